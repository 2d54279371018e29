"""The oracle on coordinate-based trees with uneven leaves (Sec. 1; Example 3 of Sec. 3).

Pins: the leaf offsets against a brute-force count in exact rational arithmetic; uniform
points must reproduce the uniform-leaf factorization bit for bit; exact mode (no sampling,
eps = 1e-15, full-rank IDs) on points with empty leaves must reproduce K; and the fully
random NUFFT of Example 3 must meet the tolerance against the dense sum, forward and adjoint.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import idbf, kernels
from paper_1809_10573_gb300 import inputs


def _product(mats):
    P = mats[0]
    for M in mats[1:]:
        P = M @ P
    return P


def test_dyadic_leaves_against_an_exact_count():
    rng = np.random.default_rng(3)
    for lo, hi, L in ((0.0, 1.0, 4), (-512.0, 512.0, 5), (-3.5, 2.25, 3)):
        p = np.sort(rng.uniform(lo, hi, 300))
        # points exactly on interior leaf edges belong to the leaf on their right
        edges = [lo + (hi - lo) * j / (1 << L) for j in range(1, 1 << L)]
        p = np.sort(np.concatenate([p, edges[::3]]))
        off = idbf.dyadic_leaves(p, lo, hi, L)
        assert off[0] == 0 and off[-1] == p.size and off.size == (1 << L) + 1
        flo, fw = Fraction(lo), Fraction(hi) - Fraction(lo)
        for j in range(1 << L):
            a, b = flo + fw * Fraction(j, 1 << L), flo + fw * Fraction(j + 1, 1 << L)
            inside = [i for i, v in enumerate(p) if a <= Fraction(v) < b]
            assert off[j + 1] - off[j] == len(inside)
            if inside:
                assert inside[0] == off[j] and inside[-1] == off[j + 1] - 1
    with pytest.raises(ValueError):
        idbf.dyadic_leaves(np.array([0.5, 0.2]), 0.0, 1.0, 2)
    with pytest.raises(ValueError):
        idbf.dyadic_leaves(np.array([0.2, 1.0]), 0.0, 1.0, 2)


def test_levels_for():
    assert idbf.levels_for(1000, 16) == 6
    assert idbf.levels_for(4096, 64) == 6
    assert idbf.levels_for(3000, 32) == 7
    assert idbf.levels_for(100, 64) == 2


def test_uniform_points_reproduce_the_uniform_factorization():
    N, n0, eps = 1024, 16, 1e-8
    x, xi = inputs.uniform_grid(N)
    L = idbf.levels_of(N, n0)
    ro = idbf.dyadic_leaves(x, 0.0, 1.0, L)
    co = idbf.dyadic_leaves(xi, -N / 2, N / 2, L)
    assert np.array_equal(ro, np.arange(0, N + 1, n0)) and np.array_equal(co, ro)
    K = kernels.Kernel(kernels.KIND_FIO, c_profile=1)
    a = idbf.export(idbf.build(K, x, xi, eps, n0))
    b = idbf.export(idbf.build(K, x, xi, eps, None, leaves=(ro, co)))
    for key in ("seg_len", "blk_rows", "blk_cols", "blk_moff", "blk_ioff", "idx", "mat"):
        assert np.array_equal(a[key], b[key]), key
    assert a["n0"] == n0 and b["n0"] == 0


def _clustered(N, seed):
    # rows only in [-N/2, N/8): the three leaves above are empty; columns avoid [0.25, 0.5)
    rng = np.random.default_rng(seed)
    om = np.sort(rng.uniform(-N / 2, N / 8, N))
    xs = np.sort(np.concatenate([rng.uniform(0.0, 0.25, N // 2), rng.uniform(0.5, 1.0, N - N // 2)]))
    return om, xs


def test_exact_mode_with_empty_leaves_reproduces_K():
    N, L = 48, 3
    om, xs = _clustered(N, 5)
    ro, co = idbf.dyadic_leaves(om, -N / 2, N / 2, L), idbf.dyadic_leaves(xs, 0.0, 1.0, L)
    assert np.sum(np.diff(ro) == 0) >= 3 and np.sum(np.diff(co) == 0) >= 2
    K = kernels.Kernel(kernels.KIND_DFT, sign=-1)
    F = idbf.build(K, om, xs, 1e-15, None, sampler="all", leaves=(ro, co))
    Kd = K.entries(om, xs, np.arange(N), np.arange(N))
    P = _product(idbf.dense_factors(F))
    assert np.linalg.norm(P - Kd) < 1e-11 * np.linalg.norm(Kd)
    g = inputs.complex_gaussian(N, 2, seed=1)
    assert idbf.relative_error(idbf.apply(F, g), Kd @ g) < 1e-12
    assert idbf.relative_error(idbf.apply_adjoint(F, g), Kd.conj().T @ g) < 1e-12


@pytest.mark.parametrize("N,n0,eps", [(1000, 16, 1e-6), (1000, 16, 1e-8), (3000, 32, 1e-6)])
def test_nufft_example3_meets_the_tolerance(N, n0, eps):
    om, xs = inputs.nufft_points(N, seed=N)
    L = idbf.levels_for(N, n0)
    ro, co = idbf.dyadic_leaves(om, -N / 2, N / 2, L), idbf.dyadic_leaves(xs, 0.0, 1.0, L)
    assert np.diff(ro).min() != np.diff(ro).max()  # uneven leaves
    K = kernels.Kernel(kernels.KIND_DFT, sign=-1)
    F = idbf.build(K, om, xs, eps, None, leaves=(ro, co))
    g = inputs.complex_gaussian(N, 1, seed=2)[:, 0]
    assert idbf.relative_error(idbf.apply(F, g), idbf.dense_matvec(K, om, xs, g)) < 10 * eps
    Kd = K.entries(om, xs, np.arange(N), np.arange(N))
    assert idbf.relative_error(idbf.apply_adjoint(F, g), Kd.conj().T @ g) < 10 * eps


def test_dense_factors_of_uneven_leaves_reproduce_apply():
    N, n0 = 300, 8
    om, xs = inputs.nufft_points(N, seed=11)
    L = idbf.levels_for(N, n0)
    F = idbf.build(kernels.Kernel(kernels.KIND_DFT, sign=-1), om, xs, 1e-7, None,
                   leaves=(idbf.dyadic_leaves(om, -N / 2, N / 2, L), idbf.dyadic_leaves(xs, 0.0, 1.0, L)))
    g = inputs.complex_gaussian(N, 1, seed=3)[:, 0]
    v = g
    for M in idbf.dense_factors(F):
        v = M @ v
    assert np.allclose(v, idbf.apply(F, g), rtol=0, atol=1e-12 * np.abs(v).max())


def test_invalid_leaf_offsets():
    N = 64
    om, xs = inputs.nufft_points(N, seed=1)
    K = kernels.Kernel(kernels.KIND_DFT)
    good = np.arange(0, N + 1, 8)
    for bad in (np.arange(0, N + 1, 16)[:4], np.r_[0, 9, 8, np.arange(24, N + 1, 8)], np.r_[good[:-1], N - 1]):
        with pytest.raises(ValueError):
            idbf.build(K, om, xs, 1e-6, None, leaves=(bad, good))


def test_example3_settings_of_the_paper():
    # Fig. N: (eps, k) = (1e-6, min{m,n}) and (1e-6, 30) give O(eps); (1e-15, 30) is near machine
    # precision. Stored entries grow like N log N (at most N log^2 N, Sec. 3).
    K = kernels.Kernel(kernels.KIND_DFT, sign=-1)
    per = []
    for N in (1000, 2000, 4000):
        om, xs = inputs.nufft_points(N, seed=N)
        L = idbf.levels_for(N, 8)
        lv = (idbf.dyadic_leaves(om, -N / 2, N / 2, L), idbf.dyadic_leaves(xs, 0.0, 1.0, L))
        g = inputs.complex_gaussian(N, 1, seed=1)[:, 0]
        ud = idbf.dense_matvec(K, om, xs, g)
        F = idbf.build(K, om, xs, 1e-6, None, leaves=lv)
        assert idbf.relative_error(idbf.apply(F, g), ud) < 1e-5
        per.append(sum(s["nnz"] for s in idbf.stats(F)) / (N * np.log2(N)))
        if N == 1000:
            F = idbf.build(K, om, xs, 1e-15, None, rank_cap=30, leaves=lv)
            assert idbf.relative_error(idbf.apply(F, g), ud) < 1e-13
            F = idbf.build(K, om, xs, 1e-6, None, rank_cap=30, leaves=lv)
            assert idbf.relative_error(idbf.apply(F, g), ud) < 1e-5
    assert max(per) / min(per) < 1.5


def test_nufft_points_generator():
    om, xs = inputs.nufft_points(1000, seed=3)
    assert om.size == xs.size == 1000
    assert om.min() >= -500 and om.max() < 500 and xs.min() >= 0 and xs.max() < 1
    assert np.all(np.diff(om) >= 0) and np.all(np.diff(xs) >= 0)
    om2, xs2 = inputs.nufft_points(1000, seed=3)
    assert np.array_equal(om, om2) and np.array_equal(xs, xs2)
    assert not np.array_equal(om, inputs.nufft_points(1000, seed=4)[0])
