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
             "IDBF_MODE_TF32X3_S64": P.MODE_TF32X3_S64, "IDBF_QR_DF64": P.QR_DF64,
             "IDBF_MODE_FP32": P.MODE_FP32, "IDBF_STORE_C64": P.STORE_C64, "IDBF_KERNEL_J0": P.KERNEL_J0,
             "IDBF_SAMPLE_ALL": P.SAMPLE_ALL}
    for name, val in pairs.items():
        assert int(defs[name]) == val, name


def test_import_validates_uneven_leaves(lib):
    # factors on coordinate-based trees with uneven leaves (Example 3) are exported with n0 = 0 and
    # leaf offsets; without the offsets the host-side validation refuses them, and offsets that do
    # not rise from 0 to N, or disagree with the blocks of the first and last levels, are refused
    # before any device work
    from oracle import idbf, kernels
    from paper_1809_10573_gb300 import inputs
    N = 96
    om, xs = inputs.nufft_points(N, seed=4)
    leaves = (idbf.dyadic_leaves(om, -N / 2, N / 2, 3), idbf.dyadic_leaves(xs, 0.0, 1.0, 3))
    ex = idbf.export(idbf.build(kernels.Kernel(kernels.KIND_DFT, sign=-1), om, xs, 1e-6, None, leaves=leaves))
    assert ex["n0"] == 0
    assert _call_import(lib, ex)[0] == _lib.EINVAL

    def with_offsets(ro, co):
        keep = [np.ascontiguousarray(ex[k]) for k in ("seg_len", "blk_rows", "blk_cols", "blk_moff", "blk_ioff", "mat", "idx")]
        ro, co = np.ascontiguousarray(ro, dtype=np.int64), np.ascontiguousarray(co, dtype=np.int64)
        f = _lib.HostFactors(ex["N"], 0, ex["L"], *[a.ctypes.data for a in keep[:5]], keep[5].ctypes.data,
                             keep[5].size, keep[6].ctypes.data, keep[6].size, ro.ctypes.data, co.ctypes.data)
        out = C.c_void_p()
        return lib.idbf_import_factors(C.byref(f), 0, None, C.byref(out))

    ro, co = ex["row_leaf_off"], ex["col_leaf_off"]
    bad = co.copy()
    bad[-1] += 1
    assert with_offsets(ro, bad) == _lib.EINVAL           # does not end at N
    bad = co.copy()
    bad[2], bad[3] = bad[3], bad[2]
    if bad[2] != bad[3]:
        assert with_offsets(ro, bad) == _lib.EINVAL       # not rising
    j = int(np.argmax(np.diff(co) > 0))
    bad = co.copy()
    bad[j + 1] -= 1                                       # leaf j one point short: level-0 blocks disagree
    assert with_offsets(ro, bad) == _lib.EFORMAT


def test_ctypes_structures_match_the_c_layout(tmp_path):
    """Sizes and field offsets of the ctypes structures equal those a C compiler gives the
    header's structures (a field added to one side only would shift every later field)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    checks = [("idbf_stats_t", _lib.Stats, ["entries", "segment_entries", "device_bytes", "level_variant",
                                            "level_storage", "boundary_entries"]),
              ("idbf_params", _lib.Params, ["leaf", "seed", "qr_arith"]),
              ("idbf_host_factors", _lib.HostFactors, ["seg_len", "mat_len", "idx_len", "col_leaf_off"]),
              ("idbf_kernel", _lib.Kernel, ["c_profile"])]
    body = []
    for cname, _, fields in checks:
        body.append(f'printf("%zu\\n", sizeof({cname}));')
        body += [f'printf("%zu\\n", offsetof({cname}, {f}));' for f in fields]
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "idbf.h"\nint main(void) {\n'
                   + "\n".join(body) + "\nreturn 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    want = []
    for _, cls, fields in checks:
        want.append(C.sizeof(cls))
        want += [getattr(cls, f).offset for f in fields]
    assert got == want


def test_dyadic_leaves_of_the_library_match_the_oracle(lib):
    """idbf_dyadic_leaves (host code of the library, no GPU) gives the oracle's coordinate-based
    leaves (Sec. 1), points on interior edges included, and refuses points outside the domain."""
    from oracle import idbf
    rng = np.random.default_rng(7)
    for lo, hi, L, n in ((0.0, 1.0, 6, 1000), (-1500.0, 1500.0, 7, 3000), (-3.5, 2.25, 3, 0), (0.0, 1.0, 2, 1)):
        p = np.sort(rng.uniform(lo, hi, n))
        if n:
            edges = lo + (hi - lo) * (np.arange(1, 1 << L, dtype=np.float64) / (1 << L))
            p = np.sort(np.concatenate([p, edges[::2]]))
        off = P.dyadic_leaves(p, lo, hi, L)
        assert np.array_equal(off, idbf.dyadic_leaves(p, lo, hi, L))
    with pytest.raises(P.IDBFError):
        P.dyadic_leaves(np.array([0.2, 1.0]), 0.0, 1.0, 2)
    with pytest.raises(P.IDBFError):
        P.dyadic_leaves(np.array([0.5, 0.2]), 0.0, 1.0, 2)


def test_tree_depth_matches_the_oracle_reading():
    from oracle import idbf
    for N, n0 in ((1000, 16), (4096, 64), (3000, 32), (100, 64), (1 << 20, 64), (12345, 8)):
        assert P.tree_depth(N, n0) == idbf.levels_for(N, n0)
