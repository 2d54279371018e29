"""The 3xTF32 tensor-core apply (tcgen05) of many right-hand sides against the oracle.

Split precision: every FP32 operand is x_hi + x_lo with x_hi = tf32(x); the three products
hi*hi + hi*lo + lo*hi accumulate in FP32, so a block product is as accurate as an FP32 one
(unit roundoff 6e-8, plus ~2^-22 from the lo parts held in TF32). Through L + 1 levels of sums of a
few hundred terms that bounds the error against the oracle's FP64 apply of the same factors by
~1e-5; the test uses 2e-5, the same bar as the FP32 CUDA-core apply."""
import numpy as np
import pytest
import torch

import paper_1809_10573_gb300 as P
from oracle import idbf
from paper_1809_10573_gb300 import inputs
from tests.cases import oracle_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.mark.parametrize("case,nrhs", [("dft_1024", 5), ("dft_1024", 130), ("fio_base_4096", 256),
                                       ("fio_base_8192_oddL", 64), ("fio_paper_2048", 17)])
def test_tf32x3_matches_oracle(case, nrhs):
    c = oracle_case(case)
    plan = P.Plan.import_factors(c["ex"], storage=P.STORE_C64)
    X = inputs.complex_gaussian(c["N"], nrhs, seed=81)
    xd = torch.from_numpy(X.astype(np.complex64)).cuda()
    y = plan.apply(xd, mode=P.MODE_TF32X3)
    plan.sync_status()
    ref = idbf.apply(c["F"], X)
    e_tc = rel(y.cpu().numpy(), ref)
    e_32 = rel(plan.apply(xd, mode=P.MODE_FP32).cpu().numpy(), ref)
    assert e_tc < 2e-5, (e_tc, e_32)


def test_tf32x3_adjoint_is_refused():
    c = oracle_case("dft_1024")
    plan = P.Plan.import_factors(c["ex"], storage=P.STORE_C64)
    xd = torch.zeros((c["N"], 2), dtype=torch.complex64, device="cuda")
    with pytest.raises(P.IDBFError):
        plan.apply_adjoint(xd, mode=P.MODE_TF32X3)


def test_tf32x3_tall_blocks_within_the_split_precision_bar():
    """GPU-built FIO at N = 2^16, eps = 1e-6: blocks of up to ~184 rows take three 64-row passes,
    and 160 right-hand sides two M tiles (the second ragged). The split-precision form must stay
    within 1e-6 + eps of the FP64 apply; against the FP64 apply of the same factors (eps does not
    enter) the test asks for 2e-6."""
    N = 1 << 16
    x, xi = inputs.uniform_grid(N)
    plan = P.Plan.build(x, xi, eps=1e-6, leaf=64, kernel="fio", c_profile=0, oversample=2, oversample_leaf=4)
    assert max(plan.stats()["level_kmax"]) > 128
    plan.set_storage(P.STORE_C128, P.STORE_C64)
    X = inputs.complex_gaussian(N, 160, seed=82)
    y64 = plan.apply(torch.from_numpy(X).cuda(), mode=P.MODE_FP64).cpu().numpy()
    ytc = plan.apply(torch.from_numpy(X.astype(np.complex64)).cuda(), mode=P.MODE_TF32X3)
    plan.sync_status()
    err = rel(ytc.cpu().numpy(), y64)
    assert err < 2e-6, err
