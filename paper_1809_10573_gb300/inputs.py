"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no arithmetic of the butterfly method: it only draws point sets and
right-hand sides with numpy's PCG64 generator so that the CUDA path and the CPU oracle
receive identical arrays.

Workloads follow the numerical examples of the paper (Sec. 3):
  * Example 1 (1D FIO): uniform grids x_i = i/N in [0,1) and xi_j = j - N/2 in [-N/2, N/2).
  * Example 3 (1D non-uniform DFT): the jittered variant below keeps the dyadic leaf
    structure of the uniform tree (each x_i stays inside its own cell) while moving every
    point by a uniform offset of at most 0.3/N; nufft_points draws the fully random points of
    Example 3 (x uniform in [0,1), omega uniform in [-N/2, N/2)), whose coordinate-based
    trees have leaves of uneven size.
Right-hand sides are complex Gaussian: real and imaginary parts i.i.d. N(0, 1).
"""
from __future__ import annotations

import numpy as np


def uniform_grid(N: int):
    """Example 1 grid: x_i = i/N (i = 0..N-1) and xi_j = j - N/2."""
    i = np.arange(N, dtype=np.float64)
    return i / N, i - N / 2


def schlomilch_grid(N: int):
    """Example 2 grid: x_k = (k-1)/N (k = 1..N) and xi_n = n pi (n = 1..N)."""
    i = np.arange(N, dtype=np.float64)
    return i / N, (i + 1.0) * np.pi


def jittered_grid(N: int, seed: int, jitter: float = 0.3):
    """x_i = i/N + U(-jitter, jitter)/N, xi_j = j - N/2 (sorted: |jitter| < 1/2)."""
    rng = np.random.default_rng(seed)
    i = np.arange(N, dtype=np.float64)
    return (i + rng.uniform(-jitter, jitter, N)) / N, i - N / 2


def nufft_points(N: int, seed: int):
    """Example 3: omega_k uniform in [-N/2, N/2) (the rows of K = exp(-2 pi i omega x)) and x_n
    uniform in [0, 1) (its columns), N of each, both sorted ascending."""
    rng = np.random.default_rng(seed)
    omega = np.sort(rng.uniform(-N / 2, N / 2, N))
    x = np.sort(rng.uniform(0.0, 1.0, N))
    return omega, x


def complex_gaussian(n: int, nrhs: int = 1, seed: int = 0, dtype=np.complex128):
    """An n x nrhs column-major block of complex Gaussian entries."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((nrhs, n)) + 1j * rng.standard_normal((nrhs, n))
    return np.asfortranarray(a.T.astype(dtype))


def sample_rows(N: int, count: int, seed: int):
    """`count` distinct row indices drawn uniformly (the 256-row error estimate of Sec. 3)."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(N, size=min(count, N), replace=False))


def uneven_batch(seed: int = 4, nops: int = 64, emin: int = 12, emax: int = 18,
                 rmin: int = 1, rmax: int = 32):
    """The uneven batch of operators: N = 2^e with e uniform in [emin, emax],
    nrhs uniform in [rmin, rmax]; the first half FIO kernels, the second half DFT kernels."""
    rng = np.random.default_rng(seed)
    es = rng.integers(emin, emax + 1, nops)
    rs = rng.integers(rmin, rmax + 1, nops)
    return [dict(N=1 << int(e), nrhs=int(r), kind="fio" if i < nops // 2 else "dft", seed=seed * 1000 + i)
            for i, (e, r) in enumerate(zip(es, rs))]
