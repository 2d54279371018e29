"""Strength of the oracle's pins: plausible mistakes, planted in the oracle on the CPU, must make
the pins fail. Each test first checks that the pin holds for the correct oracle, then plants
one mistake (a dropped term, a conjugated or transposed operand, a wrong index, a flipped sign,
a wrong solve, a shifted leaf boundary) and checks that the same pin now fails by a wide margin.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import idbf, interp, kernels
from paper_1809_10573_gb300 import inputs

N, N0, EPS = 256, 8, 1e-8


def _dft_error(F):
    """The DFT pin: K = exp(-2 pi i x xi) on x_i = i/N, xi_j = j - N/2 gives (K g)_i = (-1)^i FFT(g)_i."""
    g = inputs.complex_gaussian(N, 1, seed=21)[:, 0]
    ref = (-1.0) ** np.arange(N) * np.fft.fft(g)
    return idbf.relative_error(idbf.apply(F, g), ref)


@pytest.fixture
def dft():
    x, xi = inputs.uniform_grid(N)
    F = idbf.build(kernels.Kernel(kernels.KIND_DFT), x, xi, EPS, N0)
    assert _dft_error(F) < 10 * EPS
    return F


def _largest(blocks):
    return max(blocks.values(), key=lambda cr: cr[1].T.size)[1]


def test_a_dropped_interpolation_term_is_caught(dft):
    r = _largest(dft.V)
    assert r.T.size > 0
    r.T[:] = 0.0                                   # z = u[q] only, on one V block
    assert _dft_error(dft) > 1e3 * EPS


def test_a_conjugated_instead_of_transposed_operand_is_caught(dft):
    r = _largest(dft.U)
    r.T[:] = r.T.conj()                            # T^* w placed where T^T w belongs
    assert _dft_error(dft) > 1e3 * EPS


def test_a_swapped_skeleton_index_is_caught(dft):
    r = _largest(dft.V)
    r.q[[0, 1]] = r.q[[1, 0]]                      # two skeleton positions exchanged
    assert _dft_error(dft) > 1e3 * EPS


def test_a_middle_block_of_the_wrong_pair_is_caught(dft):
    a, b = (0, 0), (0, 1)
    if dft.S[a].shape == dft.S[b].shape:
        dft.S[a] = dft.S[b].copy()
    else:                                          # equal shapes are not guaranteed: damage instead
        dft.S[a] = dft.S[a][::-1].copy()
    assert _dft_error(dft) > 1e3 * EPS


def test_a_flipped_kernel_sign_is_caught(monkeypatch):
    x, xi = inputs.uniform_grid(N)
    K = kernels.Kernel(kernels.KIND_DFT)
    good = K.entries
    monkeypatch.setattr(K, "entries", lambda *a, **k: np.conj(good(*a, **k)))
    assert _dft_error(idbf.build(K, x, xi, EPS, N0)) > 0.5


def test_a_wrong_triangular_solve_is_caught(monkeypatch):
    # exact mode on a rank-3 matrix: the product of the factors must equal K
    rng = np.random.default_rng(5)
    A = (rng.standard_normal((64, 3)) + 1j * rng.standard_normal((64, 3))) @ \
        (rng.standard_normal((3, 64)) + 1j * rng.standard_normal((3, 64)))
    K = kernels.DenseKernel(A)
    x, xi = inputs.uniform_grid(64)

    def product():
        mats = idbf.dense_factors(idbf.build(K, x, xi, 1e-13, 4, sampler="all"))
        P = mats[0]
        for M in mats[1:]:
            P = M @ P
        return np.linalg.norm(P - A) / np.linalg.norm(A)

    assert product() < 1e-11
    solve = sla.solve_triangular
    monkeypatch.setattr(interp.sla, "solve_triangular",
                        lambda R, B, lower=False: solve(R.T, B, lower=True))   # R^T in place of R
    assert product() > 1e-3


def test_swapped_rows_and_columns_of_example_3_are_caught():
    # Eq. N sums over x_n for every omega_k: rows are the omega points, columns the x points.
    # Factorizing with the roles exchanged computes a different transform.
    n = 600
    om, xs = inputs.nufft_points(n, seed=8)
    L = idbf.levels_for(n, 16)
    ro, co = idbf.dyadic_leaves(om, -n / 2, n / 2, L), idbf.dyadic_leaves(xs, 0.0, 1.0, L)
    K = kernels.Kernel(kernels.KIND_DFT, sign=-1)
    g = inputs.complex_gaussian(n, 1, seed=9)[:, 0]
    ud = idbf.dense_matvec(K, om, xs, g)
    good = idbf.build(K, om, xs, 1e-8, None, leaves=(ro, co))
    assert idbf.relative_error(idbf.apply(good, g), ud) < 1e-7
    swapped = idbf.build(K, xs, om, 1e-8, None, leaves=(co, ro))
    assert idbf.relative_error(idbf.apply(swapped, g), ud) > 0.5
