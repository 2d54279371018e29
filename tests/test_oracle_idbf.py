"""Pins of the oracle's IDBF construction, apply and adjoint (Secs. 2.2-2.4 and 3)."""
import math

import numpy as np
import pytest

from oracle import idbf, kernels
from paper_1809_10573_gb300 import inputs


def _low_rank_kernel(N, r, seed):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((N, r)) + 1j * rng.standard_normal((N, r))
    C = rng.standard_normal((r, N)) + 1j * rng.standard_normal((r, N))
    return kernels.DenseKernel(B @ C)


@pytest.mark.parametrize("N,n0", [(64, 4), (128, 4), (64, 8)])   # L = 4, 5 (odd), 3 (odd)
def test_exact_mode_reproduces_a_low_rank_matrix(N, n0):
    # Every complementary block of a rank-3 matrix has rank 3: with no sampling and a tiny
    # tolerance every ID is exact, so the product of the L+1 factors must equal K. This pins
    # the index form of Eqs. expressUSV / expressUSV_L-1 / finishIDBF.
    K = _low_rank_kernel(N, 3, N + n0)
    x, xi = inputs.uniform_grid(N)
    F = idbf.build(K, x, xi, 1e-13, n0, sampler="all")
    mats = idbf.dense_factors(F)
    assert len(mats) == F.L + 1
    P = mats[0]
    for M in mats[1:]:
        P = M @ P
    assert np.linalg.norm(P - K.A) < 1e-11 * np.linalg.norm(K.A)
    v = inputs.complex_gaussian(N, 2, seed=1)
    assert np.linalg.norm(idbf.apply(F, v) - K.A @ v) < 1e-11 * np.linalg.norm(K.A @ v)
    assert np.linalg.norm(idbf.apply_adjoint(F, v) - K.A.conj().T @ v) < 1e-11 * np.linalg.norm(K.A.T @ v)
    # the middle blocks have the skeleton size; every ID found rank 3 or less
    assert all(r.k <= 3 for (_, r) in F.U.values()) and all(r.k <= 3 for (_, r) in F.V.values())


def test_exact_mode_dft():
    N, n0 = 64, 4
    x, xi = inputs.uniform_grid(N)
    K = kernels.Kernel(kernels.KIND_DFT)
    F = idbf.build(K, x, xi, 1e-15, n0, sampler="all")
    g = inputs.complex_gaussian(N, 1, seed=2)[:, 0]
    ref = (-1.0) ** np.arange(N) * np.fft.fft(g)
    assert idbf.relative_error(idbf.apply(F, g), ref) < 1e-12


@pytest.mark.parametrize("N,n0,eps", [(1024, 16, 1e-6), (1024, 16, 1e-8), (4096, 64, 1e-8)])
def test_dft_apply_matches_fft_to_eps(N, n0, eps):
    x, xi = inputs.uniform_grid(N)
    K = kernels.Kernel(kernels.KIND_DFT)
    F = idbf.build(K, x, xi, eps, n0)
    g = inputs.complex_gaussian(N, 1, seed=3)[:, 0]
    ref = (-1.0) ** np.arange(N) * np.fft.fft(g)
    assert idbf.relative_error(idbf.apply(F, g), ref) < 10 * eps


def test_paper_example1_settings():
    # Example 1 with the paper's own c(x), n0 = 8, t = 1: O(eps) error for
    # (eps, k) = (1e-6, min{m,n}), near machine precision for (1e-15, 30), and
    # Mock-Chebyshev rows much more accurate than random rows.
    N, n0 = 1024, 8
    x, xi = inputs.uniform_grid(N)
    K = kernels.Kernel(kernels.KIND_FIO, c_profile=1)
    g = inputs.complex_gaussian(N, 1, seed=1)[:, 0]
    ud = idbf.dense_matvec(K, x, xi, g)
    e_mock = idbf.relative_error(idbf.apply(idbf.build(K, x, xi, 1e-6, n0), g), ud)
    e_rand = idbf.relative_error(idbf.apply(idbf.build(K, x, xi, 1e-6, n0, sampler="random"), g), ud)
    e_15 = idbf.relative_error(idbf.apply(idbf.build(K, x, xi, 1e-15, n0, rank_cap=30), g), ud)
    assert e_mock < 10 * 1e-6
    assert e_rand > 100 * e_mock
    assert e_15 < 1e-13


def test_benchmark_fio_kernel_small():
    # the large-c' FIO (c = (2 + sin 2pi x sin 4pi x)/3), N = 4096, leaf 64, eps = 1e-8,
    # Mock-Chebyshev with 4x oversampling at the leaf step and 2x above it
    N, n0, eps = 4096, 64, 1e-8
    x, xi = inputs.uniform_grid(N)
    K = kernels.Kernel(kernels.KIND_FIO, c_profile=0)
    g = inputs.complex_gaussian(N, 1, seed=1)[:, 0]
    F = idbf.build(K, x, xi, eps, n0, t=2, t_leaf=4)
    ud = idbf.dense_matvec(K, x, xi, g)
    assert idbf.relative_error(idbf.apply(F, g), ud) < 10 * eps
    # the estimator of Sec. 3 on 256 sampled rows agrees with the full error
    rows = inputs.sample_rows(N, 256, seed=1)
    ua = idbf.apply(F, g)
    assert idbf.relative_error(ua[rows], ud[rows]) < 10 * eps


@pytest.fixture(scope="module")
def fio_small():
    N, n0 = 512, 8
    x, xi = inputs.jittered_grid(N, seed=9)
    K = kernels.Kernel(kernels.KIND_FIO, c_profile=1)
    F = idbf.build(K, x, xi, 1e-9, n0)
    return N, x, xi, K, F


def test_adjoint_dot_identity_and_dense(fio_small):
    N, x, xi, K, F = fio_small
    a = inputs.complex_gaussian(N, 1, seed=4)[:, 0]
    b = inputs.complex_gaussian(N, 1, seed=5)[:, 0]
    lhs = np.vdot(b, idbf.apply(F, a))
    rhs = np.vdot(idbf.apply_adjoint(F, b), a)
    Kd = K.entries(x, xi, np.arange(N), np.arange(N))
    assert abs(lhs - rhs) < 1e-13 * np.linalg.norm(a) * np.linalg.norm(b) * np.linalg.norm(Kd, 2)
    assert idbf.relative_error(idbf.apply_adjoint(F, b), Kd.conj().T @ b) < 1e-7


def test_linearity_and_multiple_rhs(fio_small):
    N, x, xi, K, F = fio_small
    X = inputs.complex_gaussian(N, 3, seed=6)
    Y = idbf.apply(F, X)
    for j in range(3):
        assert np.allclose(Y[:, j], idbf.apply(F, X[:, j]), rtol=0, atol=1e-12 * np.abs(Y).max())
    z = 2.5 * X[:, 0] - 1j * X[:, 1]
    assert np.allclose(idbf.apply(F, z), 2.5 * Y[:, 0] - 1j * Y[:, 1], atol=1e-11 * np.abs(Y).max())


def test_leaf_ranks_against_svd_brute_force():
    # the rank of each leaf row ID is close to the eps-rank of the full complementary block
    N, n0, eps = 256, 8, 1e-8
    x, xi = inputs.uniform_grid(N)
    K = kernels.Kernel(kernels.KIND_DFT)
    F = idbf.build(K, x, xi, eps, n0, t_leaf=2)
    for rho in range(N // n0):
        for kappa in (0, 1):
            blk = K.entries(x, xi, np.arange(rho * n0, (rho + 1) * n0),
                            np.arange(kappa * N // 2, (kappa + 1) * N // 2))
            sv = np.linalg.svd(blk, compute_uv=False)
            r_svd = int(np.sum(sv > eps * sv[0]))
            _, r = F.U[(1, rho, kappa)]
            assert abs(r.k - r_svd) <= 2


def test_stored_entries_scale_like_N_log_N():
    # each factor holds O(k^2 N / n0) entries (Sec. 1): entries / N per level is ~constant in N
    n0, eps = 16, 1e-6
    per_level, totals = [], []
    for e in (10, 11, 12, 13):
        N = 1 << e
        x, xi = inputs.uniform_grid(N)
        F = idbf.build(kernels.Kernel(kernels.KIND_DFT), x, xi, eps, n0)
        st = idbf.stats(F)
        per_level.append(max(s["nnz"] for s in st) / N)
        totals.append(sum(s["nnz"] for s in st) / (N * math.log2(N)))
    assert max(per_level) / min(per_level) < 1.5
    assert max(totals) / min(totals) < 1.5


def test_export_layout_reproduces_apply():
    N, n0 = 256, 8
    x, xi = inputs.uniform_grid(N)
    K = kernels.Kernel(kernels.KIND_FIO, c_profile=1)
    F = idbf.build(K, x, xi, 1e-7, n0)
    mats = idbf.dense_factors(F)
    g = inputs.complex_gaussian(N, 1, seed=8)[:, 0]
    v = g
    for M in mats:
        v = M @ v
    assert idbf.relative_error(v, idbf.apply(F, g)) < 1e-13


def test_invalid_sizes_are_rejected():
    x, xi = inputs.uniform_grid(96)
    with pytest.raises(ValueError):
        idbf.build(kernels.Kernel(), x, xi, 1e-6, 8)      # 96 / 8 is not a power of two
    x, xi = inputs.uniform_grid(16)
    with pytest.raises(ValueError):
        idbf.build(kernels.Kernel(), x, xi, 1e-6, 8)      # L = 1


def test_schlomilch_example2_meets_eps():
    # Example 2: J_0 on x_k = (k-1)/N, xi_n = n pi with k = min{m, n}. Like the benchmarked FIO
    # kernel, J_0(x xi) ~ sqrt(2/(pi x xi)) cos(x xi - pi/4) oscillates across a block, and the
    # Mock-Chebyshev samples need oversampling t = 2 (t = 4 at the leaves) to reach eps.
    N, n0, eps = 2048, 16, 1e-8
    x, xi = inputs.schlomilch_grid(N)
    K = kernels.Kernel(kernels.KIND_J0)
    F = idbf.build(K, x, xi, eps, n0, t=2, t_leaf=4)
    g = inputs.complex_gaussian(N, 2, seed=4)
    ref = K.entries(x, xi, np.arange(N), np.arange(N)) @ g
    assert idbf.relative_error(idbf.apply(F, g), ref) < 10 * eps

