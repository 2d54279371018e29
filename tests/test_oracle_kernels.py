"""Pins of the oracle's kernel entries and dense matvec against closed forms (Sec. 3)."""
import cmath
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import idbf, kernels
from paper_1809_10573_gb300 import inputs


@pytest.mark.parametrize("N", [64, 256, 1024])
def test_dft_dense_is_shifted_fft(N):
    # K = exp(-2 pi i x xi) on x_i = i/N, xi_j = j - N/2:  (K g)_i = (-1)^i FFT(g)_i
    x, xi = inputs.uniform_grid(N)
    g = inputs.complex_gaussian(N, 1, seed=N)[:, 0]
    K = kernels.Kernel(kernels.KIND_DFT, sign=-1)
    ref = (-1.0) ** np.arange(N) * np.fft.fft(g)
    assert idbf.relative_error(idbf.dense_matvec(K, x, xi, g), ref) < 1e-13
    Kp = kernels.Kernel(kernels.KIND_DFT, sign=+1)
    refp = (-1.0) ** np.arange(N) * N * np.fft.ifft(g)
    assert idbf.relative_error(idbf.dense_matvec(Kp, x, xi, g), refp) < 1e-13


def test_fio_with_zero_c_is_inverse_dft():
    N = 512
    x, xi = inputs.uniform_grid(N)
    g = inputs.complex_gaussian(N, 1, seed=3)[:, 0]
    K = kernels.Kernel(kernels.KIND_FIO, c_profile=2)
    ref = (-1.0) ** np.arange(N) * N * np.fft.ifft(g)
    assert idbf.relative_error(idbf.dense_matvec(K, x, xi, g), ref) < 1e-13


@pytest.mark.parametrize("profile,x0,c0", [
    (0, 0.25, 2.0 / 3.0),                                 # sin(pi/2) sin(pi) = 0
    (0, 0.125, (2.0 + math.sqrt(0.5)) / 3.0),             # sin(pi/4) sin(pi/2)
    (0, 0.0, 2.0 / 3.0),
    (1, 0.25, (2.0 + 0.2) / 16.0),                        # Example 1's printed c(x)
    (1, 0.75, (2.0 - 0.2) / 16.0),
])
def test_fio_entries_at_special_points(profile, x0, c0):
    K = kernels.Kernel(kernels.KIND_FIO, c_profile=profile)
    xis = np.array([-7.0, -3.0, -1.0, 0.0, 1.0, 2.0, 5.0])
    got = K.entries(np.array([x0]), xis, [0], np.arange(xis.size))[0]
    for v, xv in zip(got, xis):
        ref = cmath.exp(2j * math.pi * (x0 * xv + c0 * abs(xv)))
        assert abs(v - ref) < 1e-14


def test_block_indexing_matches_single_entries():
    N = 128
    x, xi = inputs.jittered_grid(N, seed=5)
    K = kernels.Kernel(kernels.KIND_FIO, c_profile=0)
    rows = np.array([3, 77, 5, 120])
    cols = np.array([0, 64, 127, 9, 31])
    B = K.entries(x, xi, rows, cols)
    for a, r in enumerate(rows):
        for b, c in enumerate(cols):
            cx = (2 + math.sin(2 * math.pi * x[r]) * math.sin(4 * math.pi * x[r])) / 3
            ref = cmath.exp(2j * math.pi * (x[r] * xi[c] + cx * abs(xi[c])))
            assert abs(B[a, b] - ref) < 1e-12


def test_frac_prod_keeps_low_order_bits():
    rng = np.random.default_rng(11)
    a = rng.uniform(0, 1, 200)
    b = np.round(rng.uniform(-2 ** 19, 2 ** 19, 200)) + rng.uniform(-0.3, 0.3, 200)
    got = kernels.frac_prod(a, b)
    for ai, bi, gi in zip(a, b, got):
        exact = Fraction(ai) * Fraction(bi)
        fr = exact - round(exact)
        assert abs(float(fr) - gi) < 4e-16


def test_golden_files_exist():
    here = os.path.join(os.path.dirname(__file__), "golden")
    assert os.path.exists(os.path.join(here, "splitmix64.txt"))


def test_j0_kernel_values_and_integral_representation():
    # Example 2 (Eq. S): K(x, xi) = J_0(x xi). Pinned independently of scipy's routine by
    # published values (Abramowitz and Stegun, Tables 9.1 and 9.5: J_0(1) and the first zero
    # j_{0,1}) and by Bessel's integral J_0(z) = (1/pi) int_0^pi cos(z sin t) dt, evaluated with
    # the trapezoidal rule on 4096 points (exponentially accurate for this periodic integrand).
    K = kernels.Kernel(kernels.KIND_J0)
    one = np.array([1.0])
    assert K.entries(np.array([0.0]), one, [0], [0])[0, 0] == 1.0
    assert abs(K.entries(one, one, [0], [0])[0, 0] - 0.7651976865579666) < 1e-15
    assert abs(K.entries(np.array([2.404825557695773]), one, [0], [0])[0, 0]) < 1e-15
    N = 64
    x, xi = inputs.schlomilch_grid(N)
    assert x[0] == 0.0 and x[1] == 1.0 / N and xi[0] == math.pi and xi[-1] == N * math.pi
    rows, cols = np.arange(0, N, 5), np.arange(0, N, 3)
    A = K.entries(x, xi, rows, cols)
    assert np.all(A.imag == 0)
    t = np.linspace(0.0, np.pi, 4097)
    w = np.full(t.size, np.pi / 4096)
    w[0] = w[-1] = np.pi / 8192
    Z = np.outer(x[rows], xi[cols])
    ref = (np.cos(Z[:, :, None] * np.sin(t)[None, None, :]) * w).sum(axis=2) / np.pi
    assert np.max(np.abs(A.real - ref)) < 1e-13
