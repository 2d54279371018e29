"""Degenerate shapes: the smallest factorization (L = 2: one V level, the middle level, one U
level) of a DFT whose IDs keep every column (eps = 1e-14, N = 16, n0 = 4). A third of its blocks
have no redundant columns (cols = 0: V blocks that only pass their inputs through) and a third
no rows; every kernel has a separate path for them. All apply forms must agree with the oracle,
which itself matches the closed-form DFT here, and a zero input must give an exactly zero
output."""
import numpy as np
import pytest
import torch

import paper_1809_10573_gb300 as P
from oracle import idbf, kernels
from paper_1809_10573_gb300 import inputs

N, N0, EPS = 16, 4, 1e-14


@pytest.fixture(scope="module")
def tiny():
    x, xi = inputs.uniform_grid(N)
    K = kernels.Kernel(kernels.KIND_DFT, sign=-1, c_profile=0)
    F = idbf.build(K, x, xi, EPS, N0)
    ex = idbf.export(F)
    assert F.L == 2
    assert (np.asarray(ex["blk_cols"]) == 0).any() and (np.asarray(ex["blk_rows"]) == 0).any()
    return dict(F=F, ex=ex, x=x, xi=xi, K=K)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def test_oracle_matches_the_closed_form_dft(tiny):
    # K(x, xi) = exp(-2 pi i x xi), x = i/N, xi = j - N/2: the DFT of the shifted vector
    X = inputs.complex_gaussian(N, 3, seed=5)
    j = np.arange(N) - N // 2
    dense = np.exp(-2j * np.pi * np.outer(np.arange(N) / N, j))
    assert rel(idbf.apply(tiny["F"], X), dense @ X) < 1e-12
    assert rel(idbf.apply_adjoint(tiny["F"], X), dense.conj().T @ X) < 1e-12


@pytest.mark.gpu
@pytest.mark.parametrize("nrhs", [1, 3, 16])
def test_every_mode_on_degenerate_blocks(tiny, nrhs):
    import __graft_entry__
    __graft_entry__.build()
    plan = P.Plan.import_factors(tiny["ex"], storage=P.STORE_C128)
    plan.set_storage(P.STORE_C128, P.STORE_DF64, P.STORE_C64)
    X = inputs.complex_gaussian(N, nrhs, seed=6)
    ref, ref_a = idbf.apply(tiny["F"], X), idbf.apply_adjoint(tiny["F"], X)
    x64 = torch.from_numpy(X).cuda()
    x32 = torch.from_numpy(X.astype(np.complex64)).cuda()
    for mode, xv, tol in ((P.MODE_FP64, x64, 1e-12), (P.MODE_DF64, x64, 1e-12), (P.MODE_FP32, x32, 2e-5)):
        assert rel(plan.apply(xv, mode=mode).cpu().numpy(), ref) < tol, mode
        assert rel(plan.apply_adjoint(xv, mode=mode).cpu().numpy(), ref_a) < tol, mode
        assert torch.count_nonzero(plan.apply(torch.zeros_like(xv), mode=mode)) == 0
    assert rel(plan.apply(x32, mode=P.MODE_TF32X3).cpu().numpy(), ref) < 2e-5
    plan.sync_status()


@pytest.mark.gpu
@pytest.mark.parametrize("mode,fmt,dt,tol", [(P.MODE_DF64, P.STORE_DF64, np.complex128, 1e-12),
                                             (P.MODE_FP32, P.STORE_C64, np.complex64, 2e-5),
                                             (P.MODE_FP64, P.STORE_C128, np.complex128, 1e-12)])
def test_every_variant_and_the_batch_on_degenerate_blocks(tiny, mode, fmt, dt, tol):
    import __graft_entry__
    __graft_entry__.build()
    plan = P.Plan.import_factors(tiny["ex"], storage=fmt)
    X = inputs.complex_gaussian(N, 1, seed=7)
    ref = idbf.apply(tiny["F"], X)
    xd = torch.from_numpy(X.astype(dt)).cuda()
    for v in range(P.NUM_FWD_VARIANTS):
        for pat in [[v] * 3] + ([[1, v, v]] if v >= 16 else []):  # fused pairs (0, 1) and (1, 2)
            plan.set_level_variants(mode, pat)
            assert rel(plan.apply(xd, mode=mode).cpu().numpy(), ref) < tol, f"variant {v}, pattern {pat}"
            plan.sync_status()
    plan.set_level_variants(mode, [])
    Xb = inputs.complex_gaussian(N, 5, seed=8)
    b = P.Batch([plan, plan], [1, 5], mode=mode)
    xs = [xd, torch.from_numpy(Xb.astype(dt)).cuda()]
    for tile in range(len(P.Batch.TILES)):
        try:
            b.set_tiling(tile, nodes_per_item=1)
        except P.IDBFError:
            continue
        ys = b.apply(xs)
        b.sync_status()
        assert rel(ys[0].cpu().numpy(), ref) < tol, tile
        assert rel(ys[1].cpu().numpy(), idbf.apply(tiny["F"], Xb)) < tol, tile
    b.close()
