"""The (eps, k) column ID and row ID of Sec. 2.1 (oracle; test infrastructure only).

Column ID (Lemma 2.1 and Eqs. pivotedQR2, acc, R2): a rank-revealing QR of the sampled rows,
    A_{s,:} Lambda = Q [R_1 R_2],
the numerical rank k_eps read from the diagonal of R, and
    T = R_1(1:k_eps, 1:k_eps)^{-1} R(1:k_eps, k_eps+1:n),
so that A ~ A_{:,q} [I T] Lambda^*, with q the first k_eps pivots (skeleton) and p the
remaining pivots in pivot order (redundant).

The rank-revealing QR is LAPACK's column-pivoted Householder QR (xGEQP3) through
scipy.linalg.qr(pivoting=True); the triangular solve is scipy's solve_triangular.

Rank rule. Eq. (acc) reads k_eps = min{k : R_1(k,k) <= eps R_1(1,1)}, which would keep the
first pivot that is already below the threshold. Reading adopted here: k_eps is the number of
leading pivots with |R(j,j)| > eps |R(1,1)| (one fewer), capped by the rank parameter k and
by min(|s|, n), and at least 1. A zero block gives k_eps = 1 and T = 0. A block with no columns,
or no sampled rows (an empty node of a coordinate-based tree, Sec. 1), gives k_eps = 0: no
skeleton, every column redundant, T of size 0 x n.

Row ID (end of Sec. 2.1): A ~ Lambda [I T]^* A_{q,:}. It is computed as the column ID of the
transpose, A^T ~ (A^T)_{:,q} [I T] Lambda^T, i.e. A ~ Lambda [I T]^T A_{q,:}; the row
interpolation matrix U = Lambda [I T]^T places a skeleton vector w at rows q and T^T w at
rows p.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


class IDResult:
    __slots__ = ("q", "p", "T", "k", "rdiag")

    def __init__(self, q, p, T, k, rdiag):
        self.q, self.p, self.T, self.k, self.rdiag = q, p, T, k, rdiag


def rank_from_diag(d, eps: float, kmax: int) -> int:
    """Number of leading |R(j,j)| > eps |R(1,1)|, capped at kmax, at least 1."""
    if d.size == 0 or d[0] == 0.0:
        return 1
    k = 0
    thr = eps * d[0]
    while k < min(kmax, d.size) and d[k] > thr:
        k += 1
    return max(k, 1)


def column_id(As, eps: float, kcap: int) -> IDResult:
    """(eps, k)-cID of the sampled block As (|s| x n)."""
    As = np.asarray(As, dtype=np.complex128)
    ns, n = As.shape
    if ns == 0 or n == 0:
        return IDResult(np.zeros(0, np.int64), np.arange(n, dtype=np.int64),
                        np.zeros((0, n), dtype=np.complex128), 0, np.zeros(0))
    R, P = sla.qr(As, mode="r", pivoting=True)
    d = np.abs(np.diag(R))
    kmax = min(ns, n, kcap if kcap > 0 else n)
    k = rank_from_diag(d, eps, kmax)
    if d.size == 0 or d[0] == 0.0:
        T = np.zeros((k, n - k), dtype=np.complex128)
    else:
        T = sla.solve_triangular(R[:k, :k], R[:k, k:], lower=False)
    return IDResult(np.asarray(P[:k], dtype=np.int64), np.asarray(P[k:], dtype=np.int64), T, k, d)


def row_id(As, eps: float, kcap: int) -> IDResult:
    """(eps, k)-rID of the sampled block As (m x |s|): the column ID of As^T."""
    return column_id(np.asarray(As).T, eps, kcap)
