"""Parity of the CUDA apply and adjoint with the oracle on the same (oracle-built) factors.

Tolerances: FP64 and double-float arithmetic must agree with the oracle's FP64 apply to 1e-12
relative (2-norm over the whole output block). FP32 factors and vectors carry a unit roundoff of
6e-8 per operation through L + 1 levels of sums of a few hundred terms; 2e-5 relative bounds
that with a margin and is far below the factorization tolerances tested (1e-6, 1e-8 are not
reachable in FP32; FP32 error is reported against the FP64 result)."""
import numpy as np
import pytest
import torch

import paper_1809_10573_gb300 as P
from oracle import idbf
from paper_1809_10573_gb300 import inputs
from tests.cases import CASES, oracle_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _plan(case, storage=P.STORE_C128):
    c = oracle_case(case)
    return c, P.Plan.import_factors(c["ex"], storage=storage)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("nrhs", [1, 5])
def test_fp64_apply_and_adjoint_match_oracle(case, nrhs):
    c, plan = _plan(case)
    X = inputs.complex_gaussian(c["N"], nrhs, seed=11)
    xd = torch.from_numpy(X).cuda()
    y = plan.apply(xd, mode=P.MODE_FP64).cpu().numpy()
    ya = plan.apply_adjoint(xd, mode=P.MODE_FP64).cpu().numpy()
    assert rel(y, idbf.apply(c["F"], X)) < 1e-12
    assert rel(ya, idbf.apply_adjoint(c["F"], X)) < 1e-12


@pytest.mark.parametrize("case", ["dft_1024", "fio_base_4096", "fio_base_8192_oddL", "fio_base_16384"])
@pytest.mark.parametrize("nrhs", [1, 6])
def test_df64_apply_and_adjoint_match_oracle(case, nrhs):
    c, plan = _plan(case, P.STORE_DF64)
    X = inputs.complex_gaussian(c["N"], nrhs, seed=12)
    xd = torch.from_numpy(X).cuda()
    assert rel(plan.apply(xd, mode=P.MODE_DF64).cpu().numpy(), idbf.apply(c["F"], X)) < 1e-12
    assert rel(plan.apply_adjoint(xd, mode=P.MODE_DF64).cpu().numpy(), idbf.apply_adjoint(c["F"], X)) < 1e-12


@pytest.mark.parametrize("case", ["dft_1024", "fio_base_4096"])
def test_fp32_apply_matches_oracle_to_single_precision(case):
    c, plan = _plan(case, P.STORE_C64)
    X = inputs.complex_gaussian(c["N"], 3, seed=13)
    xd = torch.from_numpy(X.astype(np.complex64)).cuda()
    assert rel(plan.apply(xd, mode=P.MODE_FP32).cpu().numpy(), idbf.apply(c["F"], X)) < 2e-5
    assert rel(plan.apply_adjoint(xd, mode=P.MODE_FP32).cpu().numpy(), idbf.apply_adjoint(c["F"], X)) < 2e-5


@pytest.mark.parametrize("case", ["fio_base_4096", "dft_jit_2048_oddL", "fio_paper_2048"])
@pytest.mark.parametrize("nrhs", [2, 16, 19])
def test_multi_rhs_register_tiles_match_oracle(case, nrhs):
    """FP64 and FP32 forward and adjoint applies with several right-hand sides run the
    register-tiled level kernels (8 right-hand sides per CTA below 16, 16 from 16 on; 19 leaves a
    ragged last block)."""
    c, plan = _plan(case)
    plan.set_storage(P.STORE_C128, P.STORE_C64)
    X = inputs.complex_gaussian(c["N"], nrhs, seed=16)
    ref = idbf.apply(c["F"], X)
    ref_a = idbf.apply_adjoint(c["F"], X)
    x64 = torch.from_numpy(X).cuda()
    assert rel(plan.apply(x64, mode=P.MODE_FP64).cpu().numpy(), ref) < 1e-12
    assert rel(plan.apply_adjoint(x64, mode=P.MODE_FP64).cpu().numpy(), ref_a) < 1e-12
    x32 = torch.from_numpy(X.astype(np.complex64)).cuda()
    assert rel(plan.apply(x32, mode=P.MODE_FP32).cpu().numpy(), ref) < 2e-5
    assert rel(plan.apply_adjoint(x32, mode=P.MODE_FP32).cpu().numpy(), ref_a) < 2e-5


def test_leading_dimension_and_preallocated_output():
    c, plan = _plan("dft_1024")
    N = c["N"]
    X = inputs.complex_gaussian(N, 3, seed=14)
    buf = torch.zeros((3, N + 7), dtype=torch.complex128, device="cuda")
    buf[:, :N] = torch.from_numpy(X.T.copy()).cuda()
    out = torch.zeros((3, N + 7), dtype=torch.complex128, device="cuda")
    torch.cuda.synchronize()
    plan.apply_raw(buf.data_ptr(), out.data_ptr(), 3, N + 7, P.MODE_FP64, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got = out[:, :N].cpu().numpy().T
    assert rel(got, idbf.apply(c["F"], X)) < 1e-12
    assert torch.all(out[:, N:] == 0)   # padding rows untouched


def test_storage_conversions_and_checkpoint(tmp_path):
    c, plan = _plan("fio_paper_2048")
    X = inputs.complex_gaussian(c["N"], 1, seed=15)
    xd = torch.from_numpy(X).cuda()
    y64 = plan.apply(xd, mode=P.MODE_FP64)
    plan.set_storage(P.STORE_DF64)                 # in place
    ydf = plan.apply(xd, mode=P.MODE_DF64)
    with pytest.raises(P.IDBFError):
        plan.apply(xd, mode=P.MODE_FP64)           # C128 no longer held
    plan.set_storage(P.STORE_DF64, P.STORE_C64)
    y32 = plan.apply(xd.to(torch.complex64), mode=P.MODE_FP32)
    assert rel(ydf.cpu().numpy(), y64.cpu().numpy()) < 1e-12
    assert rel(y32.cpu().numpy(), y64.cpu().numpy()) < 2e-5
    path = str(tmp_path / "f.idbf")
    plan.save(path)
    p2 = P.Plan.load(path)
    assert rel(p2.apply(xd, mode=P.MODE_FP64).cpu().numpy(), y64.cpu().numpy()) < 1e-13
    st = p2.stats()
    assert st["entries"] == sum(b.size for b in [c["ex"]["mat"]]) and st["L"] == c["F"].L


def test_stats_match_oracle_layout():
    c, plan = _plan("fio_base_4096")
    st = plan.stats()
    assert st["entries"] == c["ex"]["mat"].size
    assert st["index_entries"] == c["ex"]["idx"].size
    assert st["h_v"] == c["F"].hV and st["h_u"] == c["F"].hU


def test_invalid_calls_return_errors():
    c, plan = _plan("dft_1024")
    xd = torch.zeros(c["N"], dtype=torch.complex128, device="cuda")
    with pytest.raises(P.IDBFError):
        plan.apply(xd, mode=P.MODE_FP32 + 10)
    with pytest.raises(P.IDBFError):
        plan.apply_raw(xd.data_ptr(), xd.data_ptr() + 0, 1, c["N"] - 1, P.MODE_FP64, 0)  # ld < N


def test_bounded_waits_report_a_timeout_and_the_context_survives():
    # fault injection: the streaming kernels' producer issues no copies, so every consumer wait
    # runs out after 20 ms; the kernels must return, the host must read ETIMEOUT, and the next
    # apply on the same context must be exact again
    from paper_1809_10573_gb300 import _lib
    c, plan = _plan("fio_base_4096", P.STORE_DF64)
    L = _lib.lib()
    X = inputs.complex_gaussian(c["N"], 1, seed=31)
    xd = torch.from_numpy(X).cuda()
    assert L.idbf_debug_set_wait(plan._h, 20_000_000, 0) == _lib.OK
    plan.apply(xd, mode=P.MODE_DF64)   # one right-hand side: the streaming kernel
    with pytest.raises(P.IDBFError) as err:
        plan.sync_status()
    assert err.value.status == _lib.ETIMEOUT
    assert L.idbf_debug_set_wait(plan._h, 2_000_000_000, 1) == _lib.OK
    y = plan.apply(xd, mode=P.MODE_DF64)
    plan.sync_status()
    assert rel(y.cpu().numpy(), idbf.apply(c["F"], X)) < 1e-12


@pytest.mark.parametrize("case", ["fio_base_8192_oddL", "dft_jit_2048_oddL", "fio_base_16384"])
@pytest.mark.parametrize("mode,fmt,tol", [(P.MODE_DF64, P.STORE_DF64, 1e-12), (P.MODE_FP32, P.STORE_C64, 2e-5),
                                          (P.MODE_FP64, P.STORE_C128, 1e-12)])
def test_every_forward_variant_matches_oracle(case, mode, fmt, tol):
    # the autotuner may pick any variant on any level: each must give the oracle's result
    c, plan = _plan(case)
    plan.set_storage(fmt)
    X = inputs.complex_gaussian(c["N"], 1, seed=41)
    dt = torch.complex64 if mode == P.MODE_FP32 else torch.complex128
    xd = torch.from_numpy(X).to(dt).cuda()
    ref = idbf.apply(c["F"], X)
    L = c["F"].L
    for v in range(P.NUM_FWD_VARIANTS):   # FP64 runs variants 0 and 7; the streaming ones fall back to 0
        # variants 16-19 fuse levels l and l + 1: pairs (0, 1), (2, 3), ... and, shifted by one
        # level, (1, 2), (3, 4), ..., so that every pair of consecutive levels is fused once
        patterns = [[v] * (L + 1)] + ([[1] + [v] * L] if v >= 16 else [])
        for pat in patterns:
            plan.set_level_variants(mode, pat)
            y = plan.apply(xd, mode=mode)
            plan.sync_status()
            assert rel(y.cpu().numpy(), ref) < tol, f"variant {v}, pattern {pat}"
    ms = plan.autotune(mode, reps=2)
    assert ms > 0
    chosen = plan.stats()["level_variant"][fmt]
    assert all(0 <= v < P.NUM_FWD_VARIANTS for v in chosen)
    assert rel(plan.apply(xd, mode=mode).cpu().numpy(), ref) < tol
