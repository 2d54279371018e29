"""GB300 interpolative decomposition butterfly factorization (IDBF).

Python face of the C library in include/idbf.h: the construction (Secs. 2.1-2.4 of Pang, Ho and
Yang), the apply y = K x through L + 1 block-sparse factors (Eq. 1) and its adjoint, with
PyTorch used for device memory and streams. Every step of the apply runs in the library's CUDA
kernels; this module only marshals arguments.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import (KERNEL_DFT, KERNEL_FIO1D, KERNEL_J0, MODE_DF64, MODE_FP32, MODE_FP64, MODE_TF32X3,
                   MODE_TF32X3_S64, NUM_FWD_VARIANTS, QR_DF64, QR_FP64, SAMPLE_ALL, SAMPLE_MOCK_CHEBYSHEV, SAMPLE_RANDOM, STORE_C64, STORE_C128,
                   STORE_DF64, IDBFError)

__all__ = ["Plan", "Batch", "IDBFError", "apply", "IDBFApply", "kernel_matvec_rows", "dyadic_leaves", "tree_depth", "KERNEL_FIO1D", "KERNEL_DFT", "KERNEL_J0", "MODE_FP64",
           "MODE_DF64", "MODE_FP32", "MODE_TF32X3", "MODE_TF32X3_S64", "STORE_C128", "STORE_DF64", "STORE_C64",
           "SAMPLE_MOCK_CHEBYSHEV", "SAMPLE_RANDOM", "SAMPLE_ALL", "NUM_FWD_VARIANTS", "QR_FP64", "QR_DF64"]

_VEC_DTYPE = {MODE_FP64: torch.complex128, MODE_DF64: torch.complex128,
              MODE_FP32: torch.complex64, MODE_TF32X3: torch.complex64, MODE_TF32X3_S64: torch.complex64}


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _colmajor(x: torch.Tensor, N: int, dtype):
    """(N,) or (N, R) -> an (R, N) contiguous tensor whose transpose is the column-major block."""
    if x.dim() == 1:
        x = x[:, None]
    if x.shape[0] != N:
        raise ValueError(f"expected {N} rows, got {x.shape[0]}")
    if x.dtype != dtype:
        raise TypeError(f"mode expects {dtype}, got {x.dtype}")
    if not x.is_cuda:
        raise ValueError("vectors must be CUDA tensors")
    return x.t().contiguous()


class Plan:
    """A factorization resident on one GPU."""

    def __init__(self, handle: int, device: int):
        self._h = C.c_void_p(handle)
        self.device = device
        st = self.stats()
        self.N, self.n0, self.L = st["N"], st["n0"], st["L"]

    # ---- construction -------------------------------------------------------------------
    @classmethod
    def build(cls, x, xi, eps=1e-6, leaf=64, kernel="fio", c_profile=0, sign=-1, rank_cap=0,
              oversample=1.0, oversample_leaf=0.0, sampling=SAMPLE_MOCK_CHEBYSHEV, seed=0,
              storage=STORE_C128, qr_arith=QR_FP64, stream=None):
        L = _lib.lib()
        k = _lib.Kernel(_kernel_kind(kernel), sign, c_profile, 0)
        p = _lib.Params()
        L.idbf_default_params(C.byref(p))
        p.eps, p.leaf, p.rank_cap, p.oversample, p.oversample_leaf = eps, leaf, rank_cap, oversample, oversample_leaf
        p.sampling, p.seed, p.storage, p.qr_arith = sampling, seed, storage, qr_arith
        xa = np.ascontiguousarray(x, dtype=np.float64)
        xia = np.ascontiguousarray(xi, dtype=np.float64)
        out = C.c_void_p()
        st = L.idbf_build(C.byref(k), xa.ctypes.data, xia.ctypes.data, xa.size, C.byref(p),
                          _stream_ptr(stream), C.byref(out))
        _lib.check(st, "idbf_build")
        plan = cls(out.value, torch.cuda.current_device())
        plan.rank_capped = st == _lib.ERANKCAP
        return plan

    @classmethod
    def build_leaves(cls, x, xi, L, row_leaf_off, col_leaf_off, eps=1e-6, kernel="dft", c_profile=0, sign=-1,
                     rank_cap=0, oversample=1.0, oversample_leaf=0.0, sampling=SAMPLE_MOCK_CHEBYSHEV, seed=0,
                     storage=STORE_C128, qr_arith=QR_FP64, stream=None):
        """idbf_build_leaves: the construction on trees whose 2^L leaves are given by offsets."""
        L_ = _lib.lib()
        k = _lib.Kernel(_kernel_kind(kernel), sign, c_profile, 0)
        p = _lib.Params()
        L_.idbf_default_params(C.byref(p))
        p.eps, p.rank_cap, p.oversample, p.oversample_leaf = eps, rank_cap, oversample, oversample_leaf
        p.sampling, p.seed, p.storage, p.qr_arith = sampling, seed, storage, qr_arith
        xa = np.ascontiguousarray(x, dtype=np.float64)
        xia = np.ascontiguousarray(xi, dtype=np.float64)
        ro = np.ascontiguousarray(row_leaf_off, dtype=np.int64)
        co = np.ascontiguousarray(col_leaf_off, dtype=np.int64)
        if ro.size != (1 << L) + 1 or co.size != (1 << L) + 1:
            raise ValueError("2^L + 1 offsets per tree expected")
        out = C.c_void_p()
        st = L_.idbf_build_leaves(C.byref(k), xa.ctypes.data, xia.ctypes.data, xa.size, int(L), ro.ctypes.data,
                                  co.ctypes.data, C.byref(p), _stream_ptr(stream), C.byref(out))
        _lib.check(st, "idbf_build_leaves")
        plan = cls(out.value, torch.cuda.current_device())
        plan.rank_capped = st == _lib.ERANKCAP
        return plan

    @classmethod
    def import_factors(cls, ex: dict, storage=STORE_C128, stream=None):
        """Import factors given in the butterfly layout (a dict of numpy arrays)."""
        L = _lib.lib()
        keep = dict(seg_len=np.ascontiguousarray(ex["seg_len"], dtype=np.int32),
                    rows=np.ascontiguousarray(ex["blk_rows"], dtype=np.int32),
                    cols=np.ascontiguousarray(ex["blk_cols"], dtype=np.int32),
                    moff=np.ascontiguousarray(ex["blk_moff"], dtype=np.int64),
                    ioff=np.ascontiguousarray(ex["blk_ioff"], dtype=np.int64),
                    mat=np.ascontiguousarray(ex["mat"], dtype=np.complex128),
                    idx=np.ascontiguousarray(ex["idx"], dtype=np.int32))
        f = _lib.HostFactors(int(ex["N"]), int(ex["n0"]), int(ex["L"]), keep["seg_len"].ctypes.data,
                             keep["rows"].ctypes.data, keep["cols"].ctypes.data, keep["moff"].ctypes.data,
                             keep["ioff"].ctypes.data, keep["mat"].ctypes.data, keep["mat"].size,
                             keep["idx"].ctypes.data, keep["idx"].size)
        if int(ex["n0"]) == 0:  # leaves of uneven size (coordinate-based trees): pass their offsets
            keep["ro"] = np.ascontiguousarray(ex["row_leaf_off"], dtype=np.int64)
            keep["co"] = np.ascontiguousarray(ex["col_leaf_off"], dtype=np.int64)
            f.row_leaf_off, f.col_leaf_off = keep["ro"].ctypes.data, keep["co"].ctypes.data
        out = C.c_void_p()
        _lib.check(L.idbf_import_factors(C.byref(f), storage, _stream_ptr(stream), C.byref(out)),
                   "idbf_import_factors")
        return cls(out.value, torch.cuda.current_device())

    @classmethod
    def load(cls, path: str, storage=STORE_C128, stream=None):
        out = C.c_void_p()
        _lib.check(_lib.lib().idbf_load(path.encode(), storage, _stream_ptr(stream), C.byref(out)), "idbf_load")
        return cls(out.value, torch.cuda.current_device())

    def clone(self, stream=None) -> "Plan":
        """A copy of this plan with factor memory of its own (idbf_clone)."""
        out = C.c_void_p()
        _lib.check(_lib.lib().idbf_clone(self._h, _stream_ptr(stream), C.byref(out)), "idbf_clone")
        return Plan(out.value, self.device)

    def save(self, path: str):
        _lib.check(_lib.lib().idbf_save(self._h, path.encode()), "idbf_save")

    # ---- apply --------------------------------------------------------------------------
    def _run(self, fn, x, mode, out, stream):
        dt = _VEC_DTYPE.get(mode, torch.complex128)  # unknown modes are rejected by the library
        xt = _colmajor(x, self.N, dt)
        R = xt.shape[0]
        if out is None:
            yt = torch.empty((R, self.N), dtype=dt, device=xt.device)
        else:
            yt = out.t() if out.dim() == 2 else out[None, :]
            if not (yt.is_contiguous() and yt.shape == (R, self.N) and yt.dtype == dt):
                raise ValueError("out must be a column-major (N, R) block of the mode's dtype")
        _lib.check(fn(self._h, xt.data_ptr(), yt.data_ptr(), R, self.N, mode, _stream_ptr(stream)),
                   fn.__name__)
        if out is not None:
            return out
        return yt[0] if x.dim() == 1 else yt.t()

    def apply(self, x, mode=MODE_FP64, out=None, stream=None):
        """y = K x for x of shape (N,) or (N, R)."""
        return self._run(_lib.lib().idbf_apply, x, mode, out, stream)

    def apply_adjoint(self, x, mode=MODE_FP64, out=None, stream=None):
        """y = K^* x."""
        return self._run(_lib.lib().idbf_apply_adjoint, x, mode, out, stream)

    def apply_raw(self, x_ptr, y_ptr, nrhs, ld, mode, stream_ptr, adjoint=False):
        """The C call itself on raw device pointers (column-major blocks)."""
        L = _lib.lib()
        fn = L.idbf_apply_adjoint if adjoint else L.idbf_apply
        return _lib.check(fn(self._h, C.c_void_p(x_ptr), C.c_void_p(y_ptr), nrhs, ld, mode, C.c_void_p(stream_ptr)),
                          fn.__name__)

    def autotune(self, mode=MODE_DF64, reps=3, stream=None) -> float:
        """Pick the fastest forward kernel per level for `mode`; returns the summed level times (ms)."""
        ms = C.c_float()
        _lib.check(_lib.lib().idbf_autotune(self._h, mode, reps, _stream_ptr(stream), C.byref(ms)), "idbf_autotune")
        return ms.value

    def set_level_variants(self, mode, variants):
        arr = (C.c_int32 * len(variants))(*variants)
        _lib.check(_lib.lib().idbf_set_level_variants(self._h, mode, arr, len(variants)), "idbf_set_level_variants")

    def sync_status(self, stream=None):
        """Wait for the stream; raise IDBFError(ETIMEOUT) if a device-side wait gave up."""
        _lib.check(_lib.lib().idbf_sync_status(self._h, _stream_ptr(stream)), "idbf_sync_status")

    def reserve(self, nrhs: int):
        _lib.check(_lib.lib().idbf_reserve(self._h, nrhs), "idbf_reserve")

    def set_storage(self, *formats, stream=None):
        mask = 0
        for f in formats:
            mask |= 1 << f
        _lib.check(_lib.lib().idbf_set_storage(self._h, mask, _stream_ptr(stream)), "idbf_set_storage")

    def set_level_storage(self, level: int, *formats, stream=None):
        """Keep exactly `formats` on one level (apply order 0..L)."""
        mask = 0
        for f in formats:
            mask |= 1 << f
        _lib.check(_lib.lib().idbf_set_level_storage(self._h, int(level), mask, _stream_ptr(stream)),
                   "idbf_set_level_storage")

    def stats(self) -> dict:
        s = _lib.Stats()
        _lib.check(_lib.lib().idbf_stats(self._h, C.byref(s)), "idbf_stats")
        nl = s.L + 1
        return dict(N=s.N, n0=s.n0, L=s.L, h_v=s.h_v, h_u=s.h_u, storage_mask=s.storage_mask,
                    rank_saturated=s.rank_saturated, entries=s.entries, index_entries=s.index_entries,
                    level_entries=list(s.level_entries[:nl]), level_kmin=list(s.level_kmin[:nl]),
                    level_kmax=list(s.level_kmax[:nl]), segment_entries=s.segment_entries,
                    build_seconds=s.build_seconds, device_bytes=s.device_bytes,
                    level_variant={f: list(s.level_variant[f][:nl]) for f in range(3)},
                    level_storage=list(s.level_storage[:nl]),
                    boundary_entries=list(s.boundary_entries[:s.L]))

    def algorithmic_bytes(self, nrhs: int = 1, entry_bytes: int = 16, vec_bytes: int = 16) -> int:
        """Bytes one apply must move at least: every stored factor entry once, the int32
        skeleton / redundant indices once, x read and y written."""
        st = self.stats()
        return st["entries"] * entry_bytes + st["index_entries"] * 4 + 2 * self.N * nrhs * vec_bytes

    def level_bytes(self, nrhs: int = 1, entry_bytes: int = 16, vec_bytes: int = 16) -> int:
        """Bytes of one apply run level by level (one launch per level): algorithmic_bytes plus
        every intermediate boundary written by one level and read by the next."""
        st = self.stats()
        return self.algorithmic_bytes(nrhs, entry_bytes, vec_bytes) + 2 * sum(st["boundary_entries"]) * nrhs * vec_bytes

    def close(self):
        if self._h is not None and self._h.value:
            _lib.lib().idbf_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Forward applies of several plans (uneven N, their own numbers of right-hand sides) in one
    persistent kernel launch captured in a CUDA graph (idbf_batch_* in include/idbf.h)."""

    def __init__(self, plans, nrhs, mode=MODE_DF64):
        self.plans = list(plans)           # keep the plans alive as long as the batch
        self.nrhs = [int(r) for r in nrhs]
        self.mode = mode
        n = len(self.plans)
        hs = (C.c_void_p * n)(*[p._h.value for p in self.plans])
        rs = (C.c_int64 * n)(*self.nrhs)
        out = C.c_void_p()
        _lib.check(_lib.lib().idbf_batch_create(hs, n, rs, mode, C.byref(out)), "idbf_batch_create")
        self._h = out

    def _tables(self, xs, ys):
        n = len(self.plans)
        dt = _VEC_DTYPE[self.mode]
        xt = [_colmajor(x, p.N, dt) for x, p in zip(xs, self.plans)]
        if ys is None:
            yt = [torch.empty_like(t) for t in xt]
        else:
            yt = [y.t() if y.dim() == 2 else y[None, :] for y in ys]
        for t, p, r in zip(yt, self.plans, self.nrhs):
            if not (t.is_contiguous() and t.shape == (r, p.N) and t.dtype == dt):
                raise ValueError("outputs must be column-major (N, nrhs) blocks of the mode's dtype")
        xp = (C.c_void_p * n)(*[t.data_ptr() for t in xt])
        yp = (C.c_void_p * n)(*[t.data_ptr() for t in yt])
        ld = (C.c_int64 * n)(*[p.N for p in self.plans])
        return xt, yt, xp, yp, ld

    def apply(self, xs, ys=None, stream=None):
        """ys[o] = K_o xs[o]; xs[o] of shape (N_o,) or (N_o, nrhs[o])."""
        xt, yt, xp, yp, ld = self._tables(xs, ys)
        _lib.check(_lib.lib().idbf_batch_apply(self._h, xp, yp, ld, _stream_ptr(stream)), "idbf_batch_apply")
        self._keep = (xt, yt)
        if ys is not None:
            return ys
        return [t[0] if x.dim() == 1 else t.t() for t, x in zip(yt, xs)]

    def autotune(self, xs, reps=3, stream=None) -> float:
        xt, yt, xp, yp, ld = self._tables(xs, None)
        ms = C.c_float()
        _lib.check(_lib.lib().idbf_batch_autotune(self._h, xp, yp, ld, reps, _stream_ptr(stream), C.byref(ms)),
                   "idbf_batch_autotune")
        return ms.value

    # tile indices of idbf_batch_set_tiling: (right-hand sides per item, per thread, register-tile width)
    TILES = ((1, 1, 0), (4, 2, 0), (8, 2, 0), (8, 4, 0), (8, 0, 4), (16, 0, 4), (32, 0, 8), (16, 4, -1))

    def set_tiling(self, tile: int, nodes_per_item: int = 1):
        _lib.check(_lib.lib().idbf_batch_set_tiling(self._h, int(tile), int(nodes_per_item)), "idbf_batch_set_tiling")

    NO_SPLIT = (1 << 63) - 1  # idbf_batch_set_split: every operator in the persistent launch

    def set_split(self, min_separate_n: int):
        """Operators with N >= min_separate_n run through their own applies (idbf_batch_set_split)."""
        _lib.check(_lib.lib().idbf_batch_set_split(self._h, int(min_separate_n)), "idbf_batch_set_split")

    def split(self) -> dict:
        n, k = C.c_int64(), C.c_int32()
        _lib.check(_lib.lib().idbf_batch_split(self._h, C.byref(n), C.byref(k)), "idbf_batch_split")
        return dict(min_separate_n=n.value, separate_ops=k.value)

    def debug_set_wait(self, limit_ns: int, extra_target: int = 0):
        """Fault injection for tests (idbf_batch_debug_set_wait in include/idbf.h)."""
        _lib.check(_lib.lib().idbf_batch_debug_set_wait(self._h, int(limit_ns), int(extra_target)),
                   "idbf_batch_debug_set_wait")

    def info(self) -> dict:
        a, b, c, d = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        _lib.check(_lib.lib().idbf_batch_info(self._h, C.byref(a), C.byref(b), C.byref(c), C.byref(d)), "idbf_batch_info")
        return dict(rhs_per_item=a.value, nodes_per_item=b.value, items=c.value, ctas=d.value)

    def sync_status(self, stream=None):
        _lib.check(_lib.lib().idbf_batch_sync_status(self._h, _stream_ptr(stream)), "idbf_batch_sync_status")

    def close(self):
        if self._h is not None and self._h.value:
            _lib.lib().idbf_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dyadic_leaves(points, lo: float, hi: float, L: int):
    """Offsets (2^L + 1) of the leaves of the dyadic tree of depth L over [lo, hi) (Sec. 1), computed
    by the library (idbf_dyadic_leaves)."""
    p = np.ascontiguousarray(points, dtype=np.float64)
    off = np.zeros((1 << L) + 1, dtype=np.int64)
    _lib.check(_lib.lib().idbf_dyadic_leaves(p.ctypes.data, p.size, float(lo), float(hi), int(L), off.ctypes.data),
               "idbf_dyadic_leaves")
    return off


def tree_depth(N: int, n0: int) -> int:
    """Depth of a coordinate-based tree for N points with about n0 per leaf: the L whose mean leaf
    size N / 2^L is nearest to n0 on a log scale, at least 2."""
    import math
    if N < 1 or n0 < 1:
        raise ValueError("N and n0 must be positive")
    return max(2, int(round(math.log2(N / n0))))


def _kernel_kind(name: str) -> int:
    """"fio" (Example 1), "dft" (Example 3) or "j0" (Example 2, the Schloemilch expansion)."""
    kinds = {"fio": KERNEL_FIO1D, "dft": KERNEL_DFT, "j0": KERNEL_J0}
    if name not in kinds:
        raise ValueError(f"unknown kernel {name!r}: one of {sorted(kinds)}")
    return kinds[name]


def kernel_matvec_rows(x, xi, v, rows, kernel="fio", c_profile=0, sign=-1, stream=None):
    """Direct (dense) rows of K v on the GPU: the ground truth u^d of Sec. 3 at `rows`.
    x, xi: float64 CUDA tensors; v: complex128 CUDA tensor (N,); rows: int64 CUDA tensor."""
    k = _lib.Kernel(_kernel_kind(kernel), sign, c_profile, 0)
    y = torch.empty(rows.numel(), dtype=torch.complex128, device=v.device)
    for t, dt in ((x, torch.float64), (xi, torch.float64), (v, torch.complex128), (rows, torch.int64)):
        if not (t.is_cuda and t.dtype == dt and t.is_contiguous()):
            raise TypeError("kernel_matvec_rows: expected contiguous CUDA tensors of the documented dtypes")
    _lib.check(_lib.lib().idbf_kernel_matvec_rows(C.byref(k), x.data_ptr(), xi.data_ptr(), x.numel(), rows.data_ptr(),
                                                   rows.numel(), v.data_ptr(), y.data_ptr(), _stream_ptr(stream)),
               "idbf_kernel_matvec_rows")
    return y


def apply(plan: Plan, x, mode=MODE_FP64):
    """Differentiable y = K x (see IDBFApply)."""
    return IDBFApply.apply(x, plan, mode)


class IDBFApply(torch.autograd.Function):
    """y = K x with the hand-written adjoint as backward.

    PyTorch's complex autograd passes grad_y = dL/d(conj y) and expects dL/d(conj x); for the
    linear map y = K x that is grad_x = K^* grad_y, the conjugate-transpose butterfly (factors in
    reverse order, each block conjugate-transposed)."""

    @staticmethod
    def forward(ctx, x, plan, mode):
        ctx.plan, ctx.mode = plan, mode
        return plan.apply(x.detach(), mode=mode)

    @staticmethod
    def backward(ctx, gy):
        return ctx.plan.apply_adjoint(gy.contiguous(), mode=ctx.mode), None, None
