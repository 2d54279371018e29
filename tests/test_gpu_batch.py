"""An uneven batch (operators of different N and numbers of right-hand sides) in one persistent
launch captured in a CUDA graph, against the oracle and against the per-plan applies."""
import numpy as np
import pytest
import torch

import paper_1809_10573_gb300 as P
from paper_1809_10573_gb300 import _lib
from oracle import idbf
from paper_1809_10573_gb300 import inputs
from tests.cases import oracle_case

pytestmark = pytest.mark.gpu

CASES = [("dft_1024", 3), ("fio_paper_2048", 5), ("fio_base_4096", 1), ("dft_jit_2048_oddL", 7), ("fio_base_8192_oddL", 2)]


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.mark.parametrize("mode,fmt,dt,tol", [(P.MODE_DF64, P.STORE_DF64, np.complex128, 1e-12),
                                             (P.MODE_FP32, P.STORE_C64, np.complex64, 2e-5),
                                             (P.MODE_FP64, P.STORE_C128, np.complex128, 1e-12)])
def test_batch_matches_oracle_and_single_applies(mode, fmt, dt, tol):
    plans, xs, refs = [], [], []
    for k, (case, r) in enumerate(CASES):
        c = oracle_case(case)
        plans.append(P.Plan.import_factors(c["ex"], storage=fmt))
        X = inputs.complex_gaussian(c["N"], r, seed=90 + k)
        xs.append(torch.from_numpy(X.astype(dt)).cuda())
        refs.append(idbf.apply(c["F"], X))
    b = P.Batch(plans, [r for _, r in CASES], mode=mode)
    for rep in range(2):                       # graph replays
        ys = b.apply(xs)
        b.sync_status()
        for y, ref, p, x in zip(ys, refs, plans, xs):
            assert rel(y.cpu().numpy(), ref) < tol
            assert rel(y.cpu().numpy(), p.apply(x, mode=mode).cpu().numpy()) < (1e-13 if tol < 1e-9 else 1e-6)
    # every tiling the precision offers, then the autotuner's choice
    for tile in range(len(P.Batch.TILES)):
        try:
            b.set_tiling(tile, nodes_per_item=2 if tile % 2 else 1)
        except P.IDBFError as e:
            rb, _, tc = P.Batch.TILES[tile]
            max_rb = 32 if mode == P.MODE_FP32 else 16 if mode == P.MODE_FP64 else 8
            assert e.status == _lib.EUNSUPPORTED and ((tc != 0 and mode == P.MODE_DF64) or rb > max_rb)
            continue
        ys = b.apply(xs)
        b.sync_status()
        for y, ref in zip(ys, refs):
            assert rel(y.cpu().numpy(), ref) < tol, (tile, b.info())
    ms = b.autotune(xs, reps=2)
    assert ms > 0
    info = b.info()
    assert info["rhs_per_item"] in (1, 4, 8, 16, 32) and info["nodes_per_item"] in (1, 2, 4) and info["items"] > 0
    ys = b.apply(xs)
    b.sync_status()
    for y, ref in zip(ys, refs):
        assert rel(y.cpu().numpy(), ref) < tol
    b.close()


@pytest.mark.parametrize("mode,fmt,dt,tol", [(P.MODE_DF64, P.STORE_DF64, np.complex128, 1e-12),
                                             (P.MODE_FP32, P.STORE_C64, np.complex64, 2e-5)])
def test_batch_split_between_the_launch_and_separate_applies(mode, fmt, dt, tol):
    """Operators of N >= the split run through their own applies after the persistent launch: at
    every split (none, each N of the batch, all) the results match the oracle; with every operator
    split off there is no launch at all."""
    plans, xs, refs = [], [], []
    for k, (case, r) in enumerate(CASES):
        c = oracle_case(case)
        plans.append(P.Plan.import_factors(c["ex"], storage=fmt))
        X = inputs.complex_gaussian(c["N"], r, seed=50 + k)
        xs.append(torch.from_numpy(X.astype(dt)).cuda())
        refs.append(idbf.apply(c["F"], X))
    b = P.Batch(plans, [r for _, r in CASES], mode=mode)
    assert b.split() == dict(min_separate_n=P.Batch.NO_SPLIT, separate_ops=0)
    Ns = sorted({p.N for p in plans})
    for n in [P.Batch.NO_SPLIT] + Ns[::-1] + [1]:
        b.set_split(n)
        assert b.split()["separate_ops"] == sum(p.N >= n for p in plans)
        if n == 1:
            assert b.info()["items"] == 0 and b.info()["ctas"] == 0
        for rep in range(2):
            ys = b.apply(xs)
            b.sync_status()
            for y, ref in zip(ys, refs):
                assert rel(y.cpu().numpy(), ref) < tol, (n, rep)
    with pytest.raises(P.IDBFError):
        b.set_split(-1)
    b.set_split(Ns[-1])                        # a split set by hand is kept by the autotuner
    b.autotune(xs, reps=1)
    assert b.split()["min_separate_n"] == Ns[-1]
    b.set_split(0)                             # the autotuner chooses
    assert b.split()["min_separate_n"] == P.Batch.NO_SPLIT
    ms = b.autotune(xs, reps=1)
    assert ms > 0 and b.split()["min_separate_n"] in [P.Batch.NO_SPLIT] + Ns
    ys = b.apply(xs)
    b.sync_status()
    for y, ref in zip(ys, refs):
        assert rel(y.cpu().numpy(), ref) < tol
    b.close()


def test_batch_with_gpu_built_plans_of_uneven_size():
    plans, xs = [], []
    for k, (e, kind, r) in enumerate([(10, "fio", 2), (12, "dft", 9), (11, "fio", 1), (13, "dft", 4)]):
        N = 1 << e
        x, xi = inputs.uniform_grid(N) if kind == "fio" else inputs.jittered_grid(N, seed=N)
        p = P.Plan.build(x, xi, eps=1e-6, leaf=16, kernel=kind, c_profile=0, sign=-1)
        p.set_storage(P.STORE_DF64)
        plans.append(p)
        xs.append(torch.from_numpy(inputs.complex_gaussian(N, r, seed=k)).cuda())
    b = P.Batch(plans, [x.shape[1] for x in xs], mode=P.MODE_DF64)
    ys = b.apply(xs)
    b.sync_status()
    for y, p, x in zip(ys, plans, xs):
        assert rel(y.cpu().numpy(), p.apply(x, mode=P.MODE_DF64).cpu().numpy()) < 1e-13


def test_batch_wait_that_runs_out_reports_a_timeout_and_the_batch_recovers():
    # failure made on the host: the first operator's level-1 items wait for one more level-0
    # completion than there are level-0 items, so their bounded waits (20 ms) run out; the
    # status reports it, and with the target restored the same batch gives correct results
    plans, xs, refs = [], [], []
    for k, (case, r) in enumerate(CASES[:3]):
        c = oracle_case(case)
        plans.append(P.Plan.import_factors(c["ex"], storage=P.STORE_C64))
        X = inputs.complex_gaussian(c["N"], r, seed=70 + k)
        xs.append(torch.from_numpy(X.astype(np.complex64)).cuda())
        refs.append(idbf.apply(c["F"], X))
    b = P.Batch(plans, [r for _, r in CASES[:3]], mode=P.MODE_FP32)
    b.debug_set_wait(20_000_000, 1)
    b.apply(xs)
    with pytest.raises(P.IDBFError) as e:
        b.sync_status()
    assert e.value.status == _lib.ETIMEOUT
    b.debug_set_wait(2_000_000_000, 0)
    ys = b.apply(xs)
    b.sync_status()
    for y, ref in zip(ys, refs):
        assert rel(y.cpu().numpy(), ref) < 2e-5
    b.close()

