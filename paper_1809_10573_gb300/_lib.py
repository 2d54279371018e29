"""ctypes declarations of the C interface in include/idbf.h (argument marshalling only).

The shared library is built in-tree (paper_1809_10573_gb300/lib/libidbf.so) by build.py; if it
is missing, loading fails with an error: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libidbf.so")

OK, EINVAL, ENOMEM, ECUDA, ERANKCAP, ETIMEOUT, EFORMAT, EUNSUPPORTED = range(8)
KERNEL_FIO1D, KERNEL_DFT, KERNEL_J0 = 0, 1, 2
SAMPLE_MOCK_CHEBYSHEV, SAMPLE_RANDOM, SAMPLE_ALL = 0, 1, 2
STORE_C128, STORE_DF64, STORE_C64 = 0, 1, 2
QR_FP64, QR_DF64 = 0, 1
MODE_FP64, MODE_DF64, MODE_FP32, MODE_TF32X3, MODE_TF32X3_S64 = 0, 1, 2, 3, 4
NUM_FWD_VARIANTS = 20  # IDBF_NUM_FWD_VARIANTS
MAX_LEVELS = 48
NOALLOC_SCRATCH_BYTES = 64 << 20


class Kernel(C.Structure):
    _fields_ = [("kind", C.c_int32), ("sign", C.c_int32), ("c_profile", C.c_int32), ("reserved", C.c_int32)]


class Params(C.Structure):
    _fields_ = [("eps", C.c_double), ("oversample", C.c_double), ("oversample_leaf", C.c_double),
                ("leaf", C.c_int32), ("rank_cap", C.c_int32), ("sampling", C.c_int32),
                ("storage", C.c_int32), ("seed", C.c_uint64), ("qr_arith", C.c_int32), ("reserved", C.c_int32)]


class HostFactors(C.Structure):
    _fields_ = [("N", C.c_int64), ("n0", C.c_int32), ("L", C.c_int32),
                ("seg_len", C.c_void_p), ("blk_rows", C.c_void_p), ("blk_cols", C.c_void_p),
                ("blk_moff", C.c_void_p), ("blk_ioff", C.c_void_p),
                ("mat", C.c_void_p), ("mat_len", C.c_int64), ("idx", C.c_void_p), ("idx_len", C.c_int64),
                ("row_leaf_off", C.c_void_p), ("col_leaf_off", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [("N", C.c_int64), ("n0", C.c_int32), ("L", C.c_int32), ("h_v", C.c_int32), ("h_u", C.c_int32),
                ("storage_mask", C.c_uint32), ("rank_saturated", C.c_int32),
                ("entries", C.c_int64), ("index_entries", C.c_int64),
                ("level_entries", C.c_int64 * MAX_LEVELS), ("level_kmin", C.c_int32 * MAX_LEVELS),
                ("level_kmax", C.c_int32 * MAX_LEVELS), ("segment_entries", C.c_int64),
                ("build_seconds", C.c_double), ("device_bytes", C.c_int64),
                ("level_variant", (C.c_int32 * MAX_LEVELS) * 3), ("level_storage", C.c_uint32 * MAX_LEVELS),
                ("boundary_entries", C.c_int64 * MAX_LEVELS)]


_lib = None

# name -> (restype, argtypes); every function declared in include/idbf.h
SIGNATURES = {
    "idbf_default_params": (None, [C.POINTER(Params)]),
    "idbf_build": (C.c_int, [C.POINTER(Kernel), C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(Params),
                             C.c_void_p, C.POINTER(C.c_void_p)]),
    "idbf_build_leaves": (C.c_int, [C.POINTER(Kernel), C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p,
                                    C.c_void_p, C.POINTER(Params), C.c_void_p, C.POINTER(C.c_void_p)]),
    "idbf_dyadic_leaves": (C.c_int, [C.c_void_p, C.c_int64, C.c_double, C.c_double, C.c_int32, C.c_void_p]),
    "idbf_kernel_matvec_rows": (C.c_int, [C.POINTER(Kernel), C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                          C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "idbf_import_factors": (C.c_int, [C.POINTER(HostFactors), C.c_int32, C.c_void_p, C.POINTER(C.c_void_p)]),
    "idbf_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int32, C.c_void_p]),
    "idbf_apply_adjoint": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int32,
                                     C.c_void_p]),
    "idbf_apply_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int32,
                                     C.c_void_p]),
    "idbf_autotune": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.POINTER(C.c_float)]),
    "idbf_set_level_variants": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32]),
    "idbf_set_tc_split": (C.c_int, [C.c_void_p, C.c_int32]),
    "idbf_reserve": (C.c_int, [C.c_void_p, C.c_int64]),
    "idbf_sync_status": (C.c_int, [C.c_void_p, C.c_void_p]),
    "idbf_debug_set_wait": (C.c_int, [C.c_void_p, C.c_uint64, C.c_int32]),
    "idbf_set_storage": (C.c_int, [C.c_void_p, C.c_uint32, C.c_void_p]),
    "idbf_set_level_storage": (C.c_int, [C.c_void_p, C.c_int32, C.c_uint32, C.c_void_p]),
    "idbf_stats": (C.c_int, [C.c_void_p, C.POINTER(Stats)]),
    "idbf_batch_create": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.POINTER(C.c_void_p)]),
    "idbf_batch_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "idbf_batch_autotune": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p,
                                      C.POINTER(C.c_float)]),
    "idbf_batch_set_tiling": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32]),
    "idbf_batch_debug_set_wait": (C.c_int, [C.c_void_p, C.c_uint64, C.c_int32]),
    "idbf_batch_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                  C.POINTER(C.c_int32)]),
    "idbf_batch_sync_status": (C.c_int, [C.c_void_p, C.c_void_p]),
    "idbf_batch_set_split": (C.c_int, [C.c_void_p, C.c_int64]),
    "idbf_batch_split": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int32)]),
    "idbf_batch_destroy": (None, [C.c_void_p]),
    "idbf_save": (C.c_int, [C.c_void_p, C.c_char_p]),
    "idbf_load": (C.c_int, [C.c_char_p, C.c_int32, C.c_void_p, C.POINTER(C.c_void_p)]),
    "idbf_clone": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)]),
    "idbf_destroy": (None, [C.c_void_p]),
    "idbf_strerror": (C.c_char_p, [C.c_int]),
    "idbf_last_cuda_error": (C.c_char_p, []),
}


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libidbf.so is not built ({LIB_PATH}); run paper_1809_10573_gb300/build.py")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class IDBFError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        L = lib()
        msg = L.idbf_strerror(status).decode()
        cu = L.idbf_last_cuda_error().decode()
        super().__init__(f"{what}: {msg}" + (f" ({cu})" if status == ECUDA and cu else ""))
        self.status = status


def check(status: int, what: str = ""):
    if status not in (OK, ERANKCAP):
        raise IDBFError(status, what)
    return status
