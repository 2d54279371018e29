"""Parity at the benchmarked size (N = 2^20, the bench's launch configuration): the GPU-built
factorization of the FIO workload, applied by the kernels bench.py times, against the oracle's
direct matvec on 256 sampled rows (eps^a of Sec. 3), and properties that hold at any size:
double-float vs FP64 apply, FP32 vs FP64, and the adjoint identity <K x, y> = <x, K^* y>."""
import numpy as np
import pytest
import torch

import paper_1809_10573_gb300 as P
from oracle import idbf, kernels
from paper_1809_10573_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def plan2p20():
    import __graft_entry__
    __graft_entry__.build()
    N = 1 << 20
    x, xi = inputs.uniform_grid(N)
    plan = P.Plan.build(x, xi, eps=1e-6, leaf=64, kernel="fio", c_profile=0, oversample=2.0, oversample_leaf=4.0)
    plan.set_storage(P.STORE_C128, P.STORE_DF64, P.STORE_C64)
    plan.autotune(P.MODE_DF64, reps=1)
    plan.autotune(P.MODE_FP32, reps=1)
    yield N, x, xi, plan
    plan.close()


def test_full_size_sampled_rows_against_the_oracle(plan2p20):
    N, x, xi, plan = plan2p20
    g = inputs.complex_gaussian(N, 1, seed=2)[:, 0]
    gd = torch.from_numpy(g).cuda()
    rows = inputs.sample_rows(N, 256, seed=2)
    ud = idbf.dense_matvec(kernels.Kernel(kernels.KIND_FIO, c_profile=0), x, xi, g, rows=rows, chunk=32)
    y64 = plan.apply(gd, mode=P.MODE_FP64).cpu().numpy()
    ydf = plan.apply(gd, mode=P.MODE_DF64).cpu().numpy()
    y32 = plan.apply(gd.to(torch.complex64), mode=P.MODE_FP32).cpu().numpy()
    assert idbf.relative_error(y64[rows], ud) < 10 * 1e-6
    assert np.linalg.norm(ydf - y64) / np.linalg.norm(y64) < 1e-12
    assert np.linalg.norm(y32 - y64) / np.linalg.norm(y64) < 2e-5


def test_full_size_adjoint_identity(plan2p20):
    N, x, xi, plan = plan2p20
    a = torch.from_numpy(inputs.complex_gaussian(N, 1, seed=71)[:, 0]).cuda()
    b = torch.from_numpy(inputs.complex_gaussian(N, 1, seed=72)[:, 0]).cuda()
    lhs = torch.vdot(b, plan.apply(a, mode=P.MODE_DF64))
    rhs = torch.vdot(plan.apply_adjoint(b, mode=P.MODE_DF64), a)
    # ||K||_2 <= sqrt(N) for unimodular entries; rounding of the two applies is ~1e-14 relative
    bound = 1e-12 * float(torch.linalg.norm(a) * torch.linalg.norm(b)) * np.sqrt(N)
    assert abs(complex(lhs - rhs)) < bound
