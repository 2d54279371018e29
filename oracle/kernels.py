"""Kernel entries K(x, xi) for the 1D examples of Sec. 3 (oracle; test infrastructure only).

Example 1 (1D FIO):  K(x, xi) = exp(2 pi i Phi(x, xi)),  Phi = x xi + c(x) |xi|.
  c profile 0: c(x) = (2 + sin(2 pi x) sin(4 pi x)) / 3   (the large-c' variant benchmarked here)
  c profile 1: c(x) = (2 + 0.2 sin(2 pi x)) / 16           (the profile printed in Example 1)
  c profile 2: c(x) = 0                                    (reduces K to an inverse DFT)
Example 2 (Schloemilch expansion, Eq. S): K(x, xi) = J_0(x xi), with x_k = (k-1)/N and
  xi_n = n pi; J_0 from scipy.special (a library step), a real kernel held as complex128.
Example 3 (DFT type): K(x, xi) = exp(sign * 2 pi i x xi), sign = -1 by default.

Each entry is sampled individually in O(1) (the premise of Sec. 1). The phase is reduced
modulo 1 before the exponential: every product a*b is split exactly into p + e with Dekker's
two-product (T. J. Dekker, "A floating-point technique for extending the available
precision", Numer. Math. 18, 1971), so that frac(p) + e keeps full precision even when
|x xi| ~ N/2.
"""
from __future__ import annotations

import numpy as np

KIND_FIO = 0
KIND_DFT = 1
KIND_J0 = 2

_SPLIT = 134217729.0  # 2^27 + 1, Veltkamp splitting constant for binary64


def _split(a):
    c = _SPLIT * a
    hi = c - (c - a)
    return hi, a - hi


def two_prod(a, b):
    """Dekker's exact product: a*b = p + e with p = fl(a*b)."""
    p = a * b
    ah, al = _split(a)
    bh, bl = _split(b)
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def frac_prod(a, b):
    """(a*b) mod 1 in [-1/2, 1/2] + O(eps) without losing the low-order bits."""
    p, e = two_prod(a, b)
    return (p - np.rint(p)) + e


def c_profile(x, profile: int):
    if profile == 0:
        return (2.0 + np.sin(2 * np.pi * x) * np.sin(4 * np.pi * x)) / 3.0
    if profile == 1:
        return (2.0 + 0.2 * np.sin(2 * np.pi * x)) / 16.0
    if profile == 2:
        return np.zeros_like(x)
    raise ValueError("unknown c profile")


class Kernel:
    """A kernel K(x, xi) on point sets X (rows) and Omega (columns)."""

    def __init__(self, kind: int = KIND_FIO, sign: int = -1, c_profile: int = 0):
        self.kind, self.sign, self.c_profile = kind, sign, c_profile

    def phase(self, xr, xic):
        """Phase Phi(x, xi) mod 1 for the outer product of xr (rows) and xic (columns)."""
        X = np.asarray(xr, dtype=np.float64)[:, None]
        XI = np.asarray(xic, dtype=np.float64)[None, :]
        if self.kind == KIND_FIO:
            c = c_profile(X, self.c_profile)
            return frac_prod(X, XI) + frac_prod(c, np.abs(XI))
        if self.kind == KIND_DFT:
            return self.sign * frac_prod(X, XI)
        raise ValueError("unknown kernel kind")

    def entries(self, x, xi, rows, cols):
        """The block K(x[rows], xi[cols]) as a dense complex128 matrix."""
        if self.kind == KIND_J0:
            from scipy.special import j0
            X = np.asarray(x, dtype=np.float64)[np.asarray(rows)][:, None]
            XI = np.asarray(xi, dtype=np.float64)[np.asarray(cols)][None, :]
            return j0(X * XI).astype(np.complex128)
        ph = self.phase(x[np.asarray(rows)], xi[np.asarray(cols)])
        return np.exp(2j * np.pi * ph)


class DenseKernel:
    """An explicit matrix used as the kernel (for exact low-rank pins on tiny N)."""

    def __init__(self, A):
        self.A = np.asarray(A, dtype=np.complex128)

    def entries(self, x, xi, rows, cols):
        return self.A[np.ix_(np.asarray(rows), np.asarray(cols))]
