"""The allocation-free apply (idbf_apply_noalloc), called through the C interface.

For callers that must not allocate device memory during an apply, the library keeps its level
workspace in a fixed array compiled into the library. This test checks, on two calls in a row
(the array keeps the first call's contents), that the result equals the regular idbf_apply of
the same plan in the same mode, and the oracle's FP64 apply of the same factors, within that
mode's parity tolerance; and that a request larger than the array is refused before any GPU
work, as is the tensor-core mode, which the call does not offer.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_1809_10573_gb300 import _lib
from paper_1809_10573_gb300 import inputs

pytestmark = pytest.mark.gpu

# mode -> (storage, complex dtype, bar against idbf_apply in the same mode, bar against the oracle)
# FP64 and double-float: the 1e-12 FP64 parity bar; FP32: the bar of the FP32 apply's other tests
MODES = {
    _lib.MODE_FP64: (_lib.STORE_C128, np.complex128, 1e-12, 1e-12),
    _lib.MODE_DF64: (_lib.STORE_DF64, np.complex128, 1e-12, 1e-12),
    _lib.MODE_FP32: (_lib.STORE_C64, np.complex64, 1e-5, 2e-5),
}


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    return _lib.lib()


def _import(lib, case, storage=_lib.STORE_C128):
    from tests.cases import oracle_case
    ex = oracle_case(case)["ex"]
    keep = [np.ascontiguousarray(ex[k]) for k in ("seg_len", "blk_rows", "blk_cols", "blk_moff", "blk_ioff")]
    mat = np.ascontiguousarray(ex["mat"], dtype=np.complex128)
    idx = np.ascontiguousarray(ex["idx"], dtype=np.int32)
    f = _lib.HostFactors(ex["N"], ex["n0"], ex["L"], *[a.ctypes.data for a in keep],
                         mat.ctypes.data, mat.size, idx.ctypes.data, idx.size)
    plan = C.c_void_p()
    assert lib.idbf_import_factors(C.byref(f), storage, None, C.byref(plan)) == _lib.OK
    return ex["N"], plan


@pytest.mark.parametrize("mode", list(MODES), ids=["fp64", "df64", "fp32"])
@pytest.mark.parametrize("case,nrhs", [("fio_base_4096", 1), ("dft_jit_2048_oddL", 3)])
def test_noalloc_apply_matches_idbf_apply_on_two_calls(lib, case, nrhs, mode):
    from oracle import idbf
    from tests.cases import oracle_case
    storage, cdt, bar_same, bar_oracle = MODES[mode]
    N, plan = _import(lib, case, storage)
    F = oracle_case(case)["F"]
    try:
        st = torch.cuda.current_stream().cuda_stream
        for call, seed in enumerate((21, 22)):
            X = inputs.complex_gaussian(N, nrhs, seed=seed).astype(cdt)
            xt = torch.from_numpy(X.T.copy()).cuda()            # column-major N x nrhs
            y_ref = torch.empty_like(xt)
            y_na = torch.full_like(xt, float("nan"))
            assert lib.idbf_apply(plan, xt.data_ptr(), y_ref.data_ptr(), nrhs, N, mode, st) == _lib.OK
            assert lib.idbf_apply_noalloc(plan, xt.data_ptr(), y_na.data_ptr(), nrhs, N, mode, st) == _lib.OK
            torch.cuda.synchronize()
            a, b = y_na.cpu().numpy().astype(np.complex128), y_ref.cpu().numpy().astype(np.complex128)
            assert np.all(np.isfinite(a)), f"call {call}"
            assert np.linalg.norm(a - b) <= bar_same * np.linalg.norm(b), f"call {call}"
            ref = idbf.apply(F, X.astype(np.complex128)).T
            assert np.linalg.norm(a - ref) <= bar_oracle * np.linalg.norm(ref), f"call {call}"
    finally:
        lib.idbf_destroy(plan)


def test_noalloc_rejects_requests_above_the_array(lib):
    N, plan = _import(lib, "fio_base_4096")
    try:
        s = _lib.Stats()
        assert lib.idbf_stats(plan, C.byref(s)) == _lib.OK
        too_many = _lib.NOALLOC_SCRATCH_BYTES // (32 * s.segment_entries) + 1
        x = torch.zeros(N, dtype=torch.complex128, device="cuda")
        st = torch.cuda.current_stream().cuda_stream
        # refused by the size check before any pointer is touched
        assert lib.idbf_apply_noalloc(plan, x.data_ptr(), x.data_ptr(), too_many, N, _lib.MODE_FP64, st) == _lib.EUNSUPPORTED
    finally:
        lib.idbf_destroy(plan)


def test_noalloc_refuses_the_tensor_core_mode(lib):
    N, plan = _import(lib, "fio_base_4096", _lib.STORE_C64)
    try:
        x = torch.zeros(N, dtype=torch.complex64, device="cuda")
        y = torch.zeros_like(x)
        st = torch.cuda.current_stream().cuda_stream
        assert lib.idbf_apply_noalloc(plan, x.data_ptr(), y.data_ptr(), 1, N, _lib.MODE_TF32X3, st) == _lib.EINVAL
    finally:
        lib.idbf_destroy(plan)
