"""Tall blocks: a rank-250 matrix with leaves of 256 points (N = 1024, L = 2) gives V-leaf
blocks of 250 x 6 and middle blocks of 250 x 500, above the 192 rows one thread row of a
streaming-kernel team covers; those levels run the two-rows-per-thread instances of the
streaming kernel, the warp-per-node variant falls back to the per-node kernel, and the
tensor-core form runs four 64-row passes. Every forward variant, the multi-RHS and adjoint
forms and the tensor-core form must agree with the oracle, which reproduces the matrix exactly
here (no sampling, every ID keeps the full rank)."""
import numpy as np
import pytest
import torch

import paper_1809_10573_gb300 as P
from oracle import idbf, kernels
from paper_1809_10573_gb300 import inputs

N, N0, RANK = 1024, 256, 250

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tall():
    import __graft_entry__
    __graft_entry__.build()
    rng = np.random.default_rng(12)
    A = (rng.standard_normal((N, RANK)) + 1j * rng.standard_normal((N, RANK))) @ \
        (rng.standard_normal((RANK, N)) + 1j * rng.standard_normal((RANK, N))) / np.sqrt(RANK)
    x, xi = inputs.uniform_grid(N)
    F = idbf.build(kernels.DenseKernel(A), x, xi, 1e-13, N0, sampler="all")
    ex = idbf.export(F)
    assert F.L == 2 and np.asarray(ex["blk_rows"]).max() > 192
    return dict(F=F, ex=ex, A=A)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.mark.parametrize("mode,fmt,tol", [(P.MODE_DF64, P.STORE_DF64, 1e-12), (P.MODE_FP32, P.STORE_C64, 2e-5),
                                          (P.MODE_FP64, P.STORE_C128, 1e-12)])
def test_every_forward_variant_on_tall_blocks(tall, mode, fmt, tol):
    plan = P.Plan.import_factors(tall["ex"], storage=fmt)
    X = inputs.complex_gaussian(N, 1, seed=3)
    ref = idbf.apply(tall["F"], X)
    assert rel(ref, tall["A"] @ X) < 1e-12
    dt = torch.complex64 if mode == P.MODE_FP32 else torch.complex128
    xd = torch.from_numpy(X).to(dt).cuda()
    for v in range(P.NUM_FWD_VARIANTS):
        for pat in [[v] * 3] + ([[1, v, v]] if v >= 16 else []):  # fused pairs (0, 1) and (1, 2)
            plan.set_level_variants(mode, pat)
            assert rel(plan.apply(xd, mode=mode).cpu().numpy(), ref) < tol, f"variant {v}, pattern {pat}"
            plan.sync_status()
    plan.autotune(mode, reps=2)
    assert rel(plan.apply(xd, mode=mode).cpu().numpy(), ref) < tol


@pytest.mark.parametrize("nrhs", [5, 16])
def test_multi_rhs_and_adjoint_on_tall_blocks(tall, nrhs):
    plan = P.Plan.import_factors(tall["ex"], storage=P.STORE_C128)
    plan.set_storage(P.STORE_C128, P.STORE_DF64, P.STORE_C64)
    X = inputs.complex_gaussian(N, nrhs, seed=4)
    ref, ref_a = idbf.apply(tall["F"], X), idbf.apply_adjoint(tall["F"], X)
    x64 = torch.from_numpy(X).cuda()
    x32 = torch.from_numpy(X.astype(np.complex64)).cuda()
    for mode, xv, tol in ((P.MODE_FP64, x64, 1e-12), (P.MODE_DF64, x64, 1e-12), (P.MODE_FP32, x32, 2e-5)):
        assert rel(plan.apply(xv, mode=mode).cpu().numpy(), ref) < tol, mode
        assert rel(plan.apply_adjoint(xv, mode=mode).cpu().numpy(), ref_a) < tol, mode
    plan.sync_status()


def test_tensor_core_form_on_tall_blocks(tall):
    plan = P.Plan.import_factors(tall["ex"], storage=P.STORE_C64)
    X = inputs.complex_gaussian(N, 130, seed=5)   # two tiles of right-hand sides, the second ragged
    ref = idbf.apply(tall["F"], X)
    y = plan.apply(torch.from_numpy(X.astype(np.complex64)).cuda(), mode=P.MODE_TF32X3)
    plan.sync_status()
    assert rel(y.cpu().numpy(), ref) < 1e-5
