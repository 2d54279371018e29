"""IDBF construction and apply (oracle; test infrastructure only).

Notation (Sec. 2): N = n0 2^L points, m = 2^L leaves, dyadic trees T_X (rows) and T_Omega
(columns) with the root at depth 0 and the leaves at depth L. Leaf j of T_X holds the rows
ro[j] .. ro[j+1]-1 and leaf j of T_Omega the columns co[j] .. co[j+1]-1; a node at depth d is
the union of its 2^(L-d) leaves. Uniform trees (Sec. 2) have ro = co = 0, n0, 2 n0, .., N.
Sec. 1 builds the trees by dyadic partitioning of the domains of X and Omega, so for points
that are not uniformly spaced (Example 3) the leaves hold different numbers of points, some
possibly none, and N need not be n0 2^L: dyadic_leaves() gives those offsets.
A row node at depth d and a column node at depth L + 1 - d form a complementary pair (Sec. 1);
every ID below belongs to one such pair. h_V = floor(L/2) column-ID steps and h_U = L - h_V row-ID steps are taken
(Sec. 2.4 stops after L/2 steps for even L; odd L splits the steps unevenly).

Construction, in the order of the LRCS (Sec. 2.2: row IDs first, then column IDs on the
skeleton rows) repeated by recursive MSCS (Secs. 2.3-2.4), for s = 1 .. h_U:
  U step s, every (rho at depth L-s+1, kappa at depth s): row ID of K(rows, columns) with
    rows    = the rows of leaf rho (s = 1), else rhat(2rho, kappa/2) u rhat(2rho+1, kappa/2)
              (the merged leaves of the compressed tree, Sec. 2.2 and Fig. rc);
    columns = all columns of kappa (s = 1), else chat(tau, sigma) over the column nodes sigma
              at depth L-s+2 below kappa, tau the ancestor of rho at depth s-1;
    result  rhat(rho, kappa) and U(rho, kappa) = Lambda [I T]^T.
  V step s (s <= h_V), every (tau at depth s, sigma at depth L-s+1): column ID with
    columns = the columns of leaf sigma (s = 1), else chat(tau/2, 2sigma) u chat(tau/2, 2sigma+1);
    rows    = rhat(rho, kappa) over the row nodes rho at depth L-s+1 below tau, kappa the
              ancestor of sigma at depth s;
    result  chat(tau, sigma) and V(tau, sigma) = [I T] Lambda^*.
  Middle factor: for rho at depth h_V+1 and sigma at depth h_U+1,
    S(rho, sigma) = K(rhat(rho, sigma/2), chat(rho/2, sigma))  (Sec. 2.2, Eq. facA; Sec. 2.4).
This is the index form of Eqs. expressUSV, expressUSV_L-1 and finishIDBF; in
Eq. expressUSV_L-1 the last block of U^{L-1} is read as U^{L-1}_{22} and the last block of
V^{L-1} as V^{L-1}_{22} (the printed _{11} and S^{L-1}_{22} are typesetting slips), and the
product has L + 1 factors: h_V column-interpolation factors, S, and h_U row-interpolation
factors.

Apply (Eq. 1): x -> V-leaf step -> V steps 2..h_V -> S -> U steps h_U..2 -> U-leaf step, with
z(tau, sigma) = u[q] + T u[p] on the V side and t[q] += w, t[p] += T^T w on the U side.
"""
from __future__ import annotations

import math

import numpy as np

from . import interp, sampling


class IDBF:
    """Factors of K ~ U^L ... U^h S^h V^h ... V^L in the index form described above.

    n0 is the leaf size of uniform trees and None for coordinate-based trees with uneven
    leaves; ro and co are the row and column leaf offsets (m + 1 each) in both cases."""

    def __init__(self, N, n0, L, ro=None, co=None):
        self.N, self.n0, self.L = N, n0, L
        self.m = 1 << L
        self.ro = np.arange(0, N + 1, n0, dtype=np.int64) if ro is None else np.asarray(ro, np.int64)
        self.co = np.arange(0, N + 1, n0, dtype=np.int64) if co is None else np.asarray(co, np.int64)
        self.hV = L // 2
        self.hU = L - self.hV
        self.U = {}     # (s, rho, kappa) -> (rows, IDResult)
        self.V = {}     # (s, tau, sigma) -> (cols, IDResult)
        self.rhat = {}  # (s, rho, kappa) -> skeleton rows (global indices)
        self.chat = {}  # (s, tau, sigma) -> skeleton columns (global indices)
        self.S = {}     # (rho, sigma) -> dense block


def levels_of(N: int, n0: int) -> int:
    if N <= 0 or n0 <= 0 or N % n0:
        raise ValueError("N must be a positive multiple of the leaf size")
    m = N // n0
    L = int(round(math.log2(m)))
    if (1 << L) != m:
        raise ValueError("N / n0 must be a power of two")
    if L < 2:
        raise ValueError("at least two tree levels are required (N >= 4 n0)")
    return L


def dyadic_leaves(points, lo: float, hi: float, L: int):
    """Leaf offsets of the dyadic tree of depth L over the domain [lo, hi) (Sec. 1): leaf j is
    the interval [lo + (hi - lo) j / 2^L, lo + (hi - lo) (j + 1) / 2^L), and offset j is the
    number of points below its left end. `points` must be ascending and inside [lo, hi)."""
    p = np.asarray(points, dtype=np.float64)
    if p.size and (p[0] < lo or p[-1] >= hi or np.any(np.diff(p) < 0)):
        raise ValueError("points must be ascending and inside [lo, hi)")
    edges = lo + (hi - lo) * (np.arange((1 << L) + 1, dtype=np.float64) / (1 << L))
    off = np.searchsorted(p, edges, side="left").astype(np.int64)
    off[-1] = p.size
    return off


def levels_for(N: int, n0: int) -> int:
    """Tree depth for N points whose leaves should hold about n0 points: the L with N / 2^L
    nearest to n0 on a log scale, at least 2 (the reading for N that is not n0 2^L)."""
    if N <= 0 or n0 <= 0:
        raise ValueError("N and n0 must be positive")
    return max(2, int(round(math.log2(N / n0))))


def _pick(coords, cands, ns, sampler, key):
    order = np.argsort(coords[cands], kind="stable")
    c = cands[order]
    if sampler == "mock":
        sel = sampling.mock_chebyshev(coords[c], ns)
    elif sampler == "random":
        sel = sampling.random_sample(c.size, ns, key)
    elif sampler == "all":
        sel = np.arange(c.size)
    else:
        raise ValueError("unknown sampling scheme")
    return c[sel]


def build(kernel, x, xi, eps: float, n0, rank_cap: int = 0, t: float = 1,
          sampler: str = "mock", seed: int = 0, t_leaf: float = None, leaves=None) -> IDBF:
    """Construct the IDBF of K(x_i, xi_j) by the recursive MSCS of Secs. 2.2-2.4.

    rank_cap = 0 takes k = min(#rows, #columns) of each complementary block (the k = min{m,n}
    setting of Example 1); t is the oversampling factor of Sec. 2.1 (t*k sampled rows or
    columns). sampler = "all" samples every candidate (no sampling; for exact-mode checks).
    t_leaf, when given, replaces t at the leaf step s = 1, where k = n0 is the full leaf size
    and an oscillatory kernel needs more samples than k to expose its row/column space.
    leaves = (ro, co), the row and column leaf offsets of coordinate-based trees (see
    dyadic_leaves), replaces the uniform leaves of size n0 (n0 is then ignored).
    """
    t_leaf = t if t_leaf is None else t_leaf

    def nsamp(ncand, k, s):
        return min(ncand, int(math.ceil((t_leaf if s == 1 else t) * k)))

    x = np.asarray(x, dtype=np.float64)
    xi = np.asarray(xi, dtype=np.float64)
    N = x.size
    if xi.size != N:
        raise ValueError("K must be square")
    if leaves is None:
        L = levels_of(N, n0)
        F = IDBF(N, n0, L)
    else:
        ro, co = (np.asarray(a, dtype=np.int64) for a in leaves)
        m = ro.size - 1
        L = int(round(math.log2(max(m, 1))))
        if co.size != ro.size or (1 << L) != m or L < 2:
            raise ValueError("leaf offsets: 2^L + 1 entries each, L >= 2")
        for o in (ro, co):
            if o[0] != 0 or o[-1] != N or np.any(np.diff(o) < 0):
                raise ValueError("leaf offsets must rise from 0 to N")
        F = IDBF(N, None, L, ro, co)
    ro, co = F.ro, F.co
    hV, hU = F.hV, F.hU
    for s in range(1, hU + 1):
        # U step s: row IDs for (rho at depth L-s+1, kappa at depth s)
        for rho in range(1 << (L - s + 1)):
            for kappa in range(1 << s):
                if s == 1:
                    rows = np.arange(ro[rho], ro[rho + 1])
                    half = F.m >> 1
                    cands = np.arange(co[kappa * half], co[(kappa + 1) * half])
                else:
                    rows = np.concatenate([F.rhat[(s - 1, 2 * rho, kappa >> 1)],
                                           F.rhat[(s - 1, 2 * rho + 1, kappa >> 1)]])
                    sh = L - 2 * s + 2
                    tau = rho >> sh
                    cands = np.concatenate([F.chat[(s - 1, tau, sg)]
                                            for sg in range(kappa << sh, (kappa + 1) << sh)])
                k = rank_cap if rank_cap > 0 else min(rows.size, cands.size)
                key = sampling.stream_key(seed, 0, s, (rho << s) + kappa)
                cols = _pick(xi, cands, nsamp(cands.size, k, s), sampler, key)
                A = kernel.entries(x, xi, rows, cols)
                r = interp.row_id(A, eps, k)
                F.U[(s, rho, kappa)] = (rows, r)
                F.rhat[(s, rho, kappa)] = rows[r.q]
        if s > hV:
            continue
        # V step s: column IDs for (tau at depth s, sigma at depth L-s+1)
        for tau in range(1 << s):
            for sigma in range(1 << (L - s + 1)):
                if s == 1:
                    cols = np.arange(co[sigma], co[sigma + 1])
                else:
                    cols = np.concatenate([F.chat[(s - 1, tau >> 1, 2 * sigma)],
                                           F.chat[(s - 1, tau >> 1, 2 * sigma + 1)]])
                sh = L - 2 * s + 1
                kappa = sigma >> sh
                cands = np.concatenate([F.rhat[(s, rho, kappa)]
                                        for rho in range(tau << sh, (tau + 1) << sh)])
                k = rank_cap if rank_cap > 0 else min(cands.size, cols.size)
                key = sampling.stream_key(seed, 1, s, (tau << (L - s + 1)) + sigma)
                rows = _pick(x, cands, nsamp(cands.size, k, s), sampler, key)
                A = kernel.entries(x, xi, rows, cols)
                r = interp.column_id(A, eps, k)
                F.V[(s, tau, sigma)] = (cols, r)
                F.chat[(s, tau, sigma)] = cols[r.q]
    for rho in range(1 << (hV + 1)):
        for sigma in range(1 << (hU + 1)):
            F.S[(rho, sigma)] = kernel.entries(x, xi, F.rhat[(hU, rho, sigma >> 1)],
                                               F.chat[(hV, rho >> 1, sigma)])
    return F


def _as_block(x, N):
    X = np.asarray(x, dtype=np.complex128)
    if X.shape[0] != N:
        raise ValueError("x must have N rows")
    return X.reshape(N, -1)


def apply(F: IDBF, x):
    """y = U^L ... S ... V^L x (Eq. 1), level by level in natural loop order."""
    N, L, hV, hU, ro, co = F.N, F.L, F.hV, F.hU, F.ro, F.co
    X = _as_block(x, N)
    z = {}
    for sigma in range(F.m):
        xs = X[co[sigma]:co[sigma + 1]]
        for tau in (0, 1):
            _, r = F.V[(1, tau, sigma)]
            z[(tau, sigma)] = xs[r.q] + r.T @ xs[r.p]
    for s in range(2, hV + 1):
        zn = {}
        for tau in range(1 << s):
            for sigma in range(1 << (L - s + 1)):
                u = np.concatenate([z[(tau >> 1, 2 * sigma)], z[(tau >> 1, 2 * sigma + 1)]])
                _, r = F.V[(s, tau, sigma)]
                zn[(tau, sigma)] = u[r.q] + r.T @ u[r.p]
        z = zn
    w = {}
    for rho in range(1 << (hV + 1)):
        for kappa in range(1 << hU):
            w[(rho, kappa)] = sum(F.S[(rho, sg)] @ z[(rho >> 1, sg)] for sg in (2 * kappa, 2 * kappa + 1))
    for s in range(hU, 1, -1):
        wn = {}
        for rho in range(1 << (L - s + 1)):
            for kp in range(1 << (s - 1)):
                na = F.rhat[(s - 1, 2 * rho, kp)].size
                nb = F.rhat[(s - 1, 2 * rho + 1, kp)].size
                t = np.zeros((na + nb, X.shape[1]), dtype=np.complex128)
                for c in (0, 1):
                    _, r = F.U[(s, rho, 2 * kp + c)]
                    wi = w[(rho, 2 * kp + c)]
                    t[r.q] += wi
                    t[r.p] += r.T.T @ wi
                wn[(2 * rho, kp)] = t[:na]
                wn[(2 * rho + 1, kp)] = t[na:]
        w = wn
    Y = np.zeros_like(X)
    for rho in range(F.m):
        t = np.zeros((ro[rho + 1] - ro[rho], X.shape[1]), dtype=np.complex128)
        for c in (0, 1):
            _, r = F.U[(1, rho, c)]
            wi = w[(rho, c)]
            t[r.q] += wi
            t[r.p] += r.T.T @ wi
        Y[ro[rho]:ro[rho + 1]] = t
    return Y.reshape(np.shape(x)) if np.ndim(x) == 1 else Y


def apply_adjoint(F: IDBF, x):
    """y = (U^L ... S ... V^L)^* x: the factors in reverse order, each conjugate-transposed."""
    N, L, hV, hU, ro, co = F.N, F.L, F.hV, F.hU, F.ro, F.co
    X = _as_block(x, N)
    w = {}
    for rho in range(F.m):
        v = X[ro[rho]:ro[rho + 1]]
        for c in (0, 1):
            _, r = F.U[(1, rho, c)]
            w[(rho, c)] = v[r.q] + r.T.conj() @ v[r.p]
    for s in range(2, hU + 1):
        wn = {}
        for rho in range(1 << (L - s + 1)):
            for kp in range(1 << (s - 1)):
                v = np.concatenate([w[(2 * rho, kp)], w[(2 * rho + 1, kp)]])
                for c in (0, 1):
                    _, r = F.U[(s, rho, 2 * kp + c)]
                    wn[(rho, 2 * kp + c)] = v[r.q] + r.T.conj() @ v[r.p]
        w = wn
    z = {}
    for tau in range(1 << hV):
        for sigma in range(1 << (hU + 1)):
            z[(tau, sigma)] = sum(F.S[(rho, sigma)].conj().T @ w[(rho, sigma >> 1)]
                                  for rho in (2 * tau, 2 * tau + 1))
    for s in range(hV, 1, -1):
        zn = {}
        for tp in range(1 << (s - 1)):
            for sigma in range(1 << (L - s + 1)):
                na = F.chat[(s - 1, tp, 2 * sigma)].size
                nb = F.chat[(s - 1, tp, 2 * sigma + 1)].size
                u = np.zeros((na + nb, X.shape[1]), dtype=np.complex128)
                for c in (0, 1):
                    _, r = F.V[(s, 2 * tp + c, sigma)]
                    zi = z[(2 * tp + c, sigma)]
                    u[r.q] += zi
                    u[r.p] += r.T.conj().T @ zi
                zn[(tp, 2 * sigma)] = u[:na]
                zn[(tp, 2 * sigma + 1)] = u[na:]
        z = zn
    Y = np.zeros_like(X)
    for sigma in range(F.m):
        u = np.zeros((co[sigma + 1] - co[sigma], X.shape[1]), dtype=np.complex128)
        for tau in (0, 1):
            _, r = F.V[(1, tau, sigma)]
            zi = z[(tau, sigma)]
            u[r.q] += zi
            u[r.p] += r.T.conj().T @ zi
        Y[co[sigma]:co[sigma + 1]] = u
    return Y.reshape(np.shape(x)) if np.ndim(x) == 1 else Y


def dense_matvec(kernel, x, xi, v, rows=None, chunk: int = 256):
    """Ground truth y = K v (or its rows `rows`), O(N^2), evaluated in row chunks."""
    x = np.asarray(x, dtype=np.float64)
    xi = np.asarray(xi, dtype=np.float64)
    V = np.asarray(v, dtype=np.complex128).reshape(xi.size, -1)
    rows = np.arange(x.size) if rows is None else np.asarray(rows)
    cols = np.arange(xi.size)
    out = np.empty((rows.size, V.shape[1]), dtype=np.complex128)
    for a in range(0, rows.size, chunk):
        out[a:a + chunk] = kernel.entries(x, xi, rows[a:a + chunk], cols) @ V
    return out.reshape(-1) if np.ndim(v) == 1 else out


def relative_error(ua, ud) -> float:
    """eps^a of Sec. 3: sqrt(sum |u^a - u^d|^2 / sum |u^d|^2) over the given entries."""
    ua = np.asarray(ua)
    ud = np.asarray(ud)
    return float(np.sqrt(np.sum(np.abs(ua - ud) ** 2) / np.sum(np.abs(ud) ** 2)))


def dense_factors(F: IDBF):
    """The L+1 sparse factors as dense N_out x N_in matrices, in apply order (tiny N only).

    Index spaces: level boundaries hold the concatenation of all segments in the butterfly
    numbering of export(); the product of the returned matrices (last @ ... @ first) is the
    IDBF approximation of K.
    """
    ex = export(F)
    L, m, ro, co = F.L, F.m, F.ro, F.co
    seg_len = ex["seg_len"]
    mats = []
    offs = [np.concatenate([[0], np.cumsum(seg_len[b])]) for b in range(L)]
    for lev in range(L + 1):
        nin = F.N if lev == 0 else int(offs[lev - 1][-1])
        nout = F.N if lev == L else int(offs[lev][-1])
        M = np.zeros((nout, nin), dtype=np.complex128)
        H = 1 << (L - lev)
        for j in range(m):
            if lev == 0:
                in_idx = np.arange(co[j], co[j + 1])
            else:
                a, b = 2 * j, 2 * j + 1
                in_idx = np.concatenate([np.arange(offs[lev - 1][a], offs[lev - 1][a + 1]),
                                         np.arange(offs[lev - 1][b], offs[lev - 1][b + 1])])
            if lev == L:
                out_idx = [np.arange(ro[j], ro[j + 1])]
            else:
                o = [(j // H) * 2 * H + (j % H) + c * H for c in (0, 1)]
                out_idx = [np.arange(offs[lev][oc], offs[lev][oc + 1]) for oc in o]
            kind = ex["level_kind"][lev]
            for c in (0, 1):
                r, cc = ex["blk_rows"][lev, j, c], ex["blk_cols"][lev, j, c]
                mo, io = ex["blk_moff"][lev, j, c], ex["blk_ioff"][lev, j, c]
                B = ex["mat"][mo:mo + r * cc].reshape(r, cc)
                if kind == 0:  # gather form: out_c = u[q] + B u[p]
                    q = ex["idx"][io:io + r]
                    p = ex["idx"][io + r:io + r + cc]
                    blk = np.zeros((r, in_idx.size), dtype=np.complex128)
                    blk[np.arange(r), q] = 1.0
                    blk[:, p] += B
                    M[np.ix_(out_idx[c], in_idx)] += blk
                elif kind == 1:  # dense: out_c = B u
                    M[np.ix_(out_idx[c], in_idx)] += B
                else:  # scatter form: t[q] += in_c, t[p] += B in_c
                    q = ex["idx"][io:io + cc]
                    p = ex["idx"][io + cc:io + cc + r]
                    tl = np.concatenate(out_idx)
                    seg_in = np.arange(offs[lev - 1][2 * j + c], offs[lev - 1][2 * j + c + 1])
                    blk = np.zeros((tl.size, seg_in.size), dtype=np.complex128)
                    blk[q, np.arange(cc)] = 1.0
                    blk[p, :] += B
                    M[np.ix_(tl, seg_in)] += blk
        mats.append(M)
    return mats


def export(F: IDBF):
    """The factors in the flat butterfly layout of the C interface (include/idbf.h).

    Level l = 0..L in apply order: l < h_V column-ID levels (gather form, kind 0), l = h_V the
    middle factor (dense, kind 1), l > h_V row-ID levels (scatter form, kind 2). Level l has
    m nodes; node j reads segments 2j and 2j+1 of boundary l-1 (leaf j of x at l = 0) and
    writes segments (j // H) 2H + j % H + c H, c = 0, 1, of boundary l with H = 2^(L-l)
    (leaf j of y at l = L). Each node has two blocks, c = 0, 1:
      kind 0: out_c = u[q_c] + M_c u[p_c], u = concat(in_0, in_1); M_c is |q_c| x |p_c|
      kind 1: out_c = M_c u
      kind 2: t[q_c] += in_c and t[p_c] += M_c in_c, t = concat(out_0, out_1); M_c = T_c^T
    Matrices are row-major complex128; idx holds q_c then p_c (int32). Leaf j of x is
    x[col_leaf_off[j] : col_leaf_off[j+1]] and leaf j of y is y[row_leaf_off[j] : row_leaf_off[j+1]];
    n0 is 0 for uneven leaves (a layout the C interface, which takes leaves of n0 entries, does
    not accept).
    """
    L, m, hV, hU = F.L, F.m, F.hV, F.hU
    n0 = F.n0 if F.n0 is not None else 0
    seg_len = np.zeros((L, 2 * m), dtype=np.int32)
    for b in range(L):
        if b < hV:
            s = b + 1
            for tau in range(1 << s):
                for sigma in range(1 << (L - s + 1)):
                    seg_len[b, (tau << (L - s + 1)) + sigma] = F.chat[(s, tau, sigma)].size
        else:
            s = hU - (b - hV)  # skeleton rows rhat(s, rho, kappa), rho at depth L-s+1
            for rho in range(1 << (L - s + 1)):
                for kappa in range(1 << s):
                    seg_len[b, (rho << s) + kappa] = F.rhat[(s, rho, kappa)].size
    rows = np.zeros((L + 1, m, 2), dtype=np.int32)
    cols = np.zeros((L + 1, m, 2), dtype=np.int32)
    moff = np.zeros((L + 1, m, 2), dtype=np.int64)
    ioff = np.zeros((L + 1, m, 2), dtype=np.int64)
    kinds = np.zeros(L + 1, dtype=np.int32)
    mats, idxs = [], []
    mo = io = 0

    def put(lev, j, c, M, idx):
        nonlocal mo, io
        rows[lev, j, c], cols[lev, j, c] = M.shape
        moff[lev, j, c], ioff[lev, j, c] = mo, io
        mats.append(np.ascontiguousarray(M).reshape(-1))
        idxs.append(np.asarray(idx, dtype=np.int32))
        mo += M.size
        io += len(idx)

    for lev in range(L + 1):
        if lev < hV:
            kinds[lev] = 0
            s = lev + 1
            for j in range(m):
                tp, sigma = j >> (L - s + 1), j & ((1 << (L - s + 1)) - 1)
                for c in (0, 1):
                    _, r = F.V[(s, 2 * tp + c, sigma)] if s > 1 else F.V[(1, c, j)]
                    put(lev, j, c, r.T, np.concatenate([r.q, r.p]))
        elif lev == hV:
            kinds[lev] = 1
            for j in range(m):
                tau, kappa = j >> hU, j & ((1 << hU) - 1)
                for c in (0, 1):
                    rho = 2 * tau + c
                    M = np.hstack([F.S[(rho, 2 * kappa)], F.S[(rho, 2 * kappa + 1)]])
                    put(lev, j, c, M, [])
        else:
            kinds[lev] = 2
            s = hU - (lev - hV - 1)
            for j in range(m):
                rho, kp = j >> (s - 1), j & ((1 << (s - 1)) - 1)
                for c in (0, 1):
                    _, r = F.U[(s, rho, 2 * kp + c)] if s > 1 else F.U[(1, j, c)]
                    put(lev, j, c, r.T.T, np.concatenate([r.q, r.p]))
    return dict(N=F.N, n0=n0, L=L, hV=hV, hU=hU, seg_len=seg_len, level_kind=kinds,
                row_leaf_off=F.ro.copy(), col_leaf_off=F.co.copy(),
                blk_rows=rows, blk_cols=cols, blk_moff=moff, blk_ioff=ioff,
                mat=np.concatenate(mats) if mats else np.zeros(0, np.complex128),
                idx=np.concatenate(idxs) if idxs else np.zeros(0, np.int32))


def stats(F: IDBF):
    """Per-level ranks and stored entries (T blocks and S; the identity part is not stored)."""
    out = []
    for s in range(1, F.hV + 1):
        ks = [r.k for (ss, _, _), (_, r) in F.V.items() if ss == s]
        ent = sum(r.T.size for (ss, _, _), (_, r) in F.V.items() if ss == s)
        out.append(dict(side="V", step=s, kmin=min(ks), kmax=max(ks), entries=ent, nnz=ent + sum(ks)))
    ent = sum(b.size for b in F.S.values())
    out.append(dict(side="S", step=0, kmin=0, kmax=0, entries=ent, nnz=ent))
    for s in range(F.hU, 0, -1):
        ks = [r.k for (ss, _, _), (_, r) in F.U.items() if ss == s]
        ent = sum(r.T.size for (ss, _, _), (_, r) in F.U.items() if ss == s)
        out.append(dict(side="U", step=s, kmin=min(ks), kmax=max(ks), entries=ent, nnz=ent + sum(ks)))
    return out
