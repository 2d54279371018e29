"""The C interface: the library loads and exports every function include/idbf.h declares, and
the host-side validation rejects bad input without touching a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import paper_1809_10573_gb300 as P
from paper_1809_10573_gb300 import _lib

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "idbf.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(idbf_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return _lib.lib()


def test_every_declared_function_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_lib.SIGNATURES), "binding and header disagree"


def test_default_params_and_strerror(lib):
    p = _lib.Params()
    lib.idbf_default_params(C.byref(p))
    assert p.eps == 1e-6 and p.leaf == 64 and p.oversample == 1.0 and p.rank_cap == 0
    for s in range(8):
        assert lib.idbf_strerror(s)


def _tiny_factors():
    from tests.cases import oracle_case
    from oracle import idbf, kernels
    from paper_1809_10573_gb300 import inputs
    x, xi = inputs.uniform_grid(64)
    F = idbf.build(kernels.Kernel(kernels.KIND_DFT), x, xi, 1e-8, 8)
    return idbf.export(F)


def _call_import(lib, ex):
    keep = [np.ascontiguousarray(ex[k]) for k in ("seg_len", "blk_rows", "blk_cols", "blk_moff", "blk_ioff", "mat", "idx")]
    f = _lib.HostFactors(ex["N"], ex["n0"], ex["L"], *[a.ctypes.data for a in keep[:5]],
                         keep[5].ctypes.data, keep[5].size, keep[6].ctypes.data, keep[6].size)
    out = C.c_void_p()
    return lib.idbf_import_factors(C.byref(f), 0, None, C.byref(out)), keep


def test_import_validation_rejects_inconsistent_factors(lib):
    ex = _tiny_factors()
    bad = dict(ex)
    bad["N"] = ex["N"] + 1
    assert _call_import(lib, bad)[0] == _lib.EINVAL
    bad = dict(ex)
    bad["idx"] = ex["idx"].copy()
    bad["idx"][0] = bad["idx"][1]            # q_0 no longer a permutation part
    assert _call_import(lib, bad)[0] == _lib.EFORMAT
    bad = dict(ex)
    bad["seg_len"] = ex["seg_len"].copy()
    bad["seg_len"][0, 3] += 1                # a segment length that no block produces
    assert _call_import(lib, bad)[0] == _lib.EFORMAT
    bad = dict(ex)
    bad["blk_moff"] = ex["blk_moff"].copy()
    nz = np.argwhere(ex["blk_rows"] * ex["blk_cols"] > 0)[0]
    bad["blk_moff"][tuple(nz)] = ex["mat"].size   # a non-empty block past the end of mat
    assert _call_import(lib, bad)[0] == _lib.EFORMAT


def test_null_arguments(lib):
    out = C.c_void_p()
    assert lib.idbf_import_factors(None, 0, None, C.byref(out)) == _lib.EINVAL
    assert lib.idbf_apply(None, None, None, 1, 1, 0, None) == _lib.EINVAL
    assert lib.idbf_stats(None, None) == _lib.EINVAL
    lib.idbf_destroy(None)


def test_python_constants_match_the_header():
    src = open(HEADER).read()
    defs = dict(re.findall(r"#define (IDBF_[A-Z0-9_]+) (\d+)\b", src))
    pairs = {"IDBF_NUM_FWD_VARIANTS": P.NUM_FWD_VARIANTS, "IDBF_MODE_TF32X3": P.MODE_TF32X3,
             "IDBF_MODE_FP32": P.MODE_FP32, "IDBF_STORE_C64": P.STORE_C64, "IDBF_KERNEL_J0": P.KERNEL_J0,
             "IDBF_SAMPLE_ALL": P.SAMPLE_ALL}
    for name, val in pairs.items():
        assert int(defs[name]) == val, name


def test_import_refuses_uneven_leaves(lib):
    # factors on coordinate-based trees with uneven leaves (Example 3) are exported with n0 = 0:
    # the C layout takes leaves of n0 entries, so the host-side validation refuses them
    from oracle import idbf, kernels
    from paper_1809_10573_gb300 import inputs
    N = 96
    om, xs = inputs.nufft_points(N, seed=4)
    leaves = (idbf.dyadic_leaves(om, -N / 2, N / 2, 3), idbf.dyadic_leaves(xs, 0.0, 1.0, 3))
    ex = idbf.export(idbf.build(kernels.Kernel(kernels.KIND_DFT, sign=-1), om, xs, 1e-6, None, leaves=leaves))
    assert ex["n0"] == 0
    assert _call_import(lib, ex)[0] == _lib.EINVAL
