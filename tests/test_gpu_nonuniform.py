"""Example 3 on the GPU: factors on coordinate-based dyadic trees (Sec. 1) whose leaves hold
uneven numbers of points, some none, applied through the C interface and compared element-wise
with the oracle's apply of the same factors.

Cases: the fully random NUFFT of Example 3 (omega uniform in [-N/2, N/2), x uniform in [0, 1),
K = exp(-2 pi i omega x)) at N = 1000 and 3000, which are not n0 2^L, and points clustered so
that whole leaves are empty (zero-length segments, blocks with no columns, exact mode). Bars:
1e-12 relative for FP64 and double-float, 2e-5 for FP32, as for the uniform cases."""
import functools

import numpy as np
import pytest
import torch

import paper_1809_10573_gb300 as P
from oracle import idbf, kernels
from paper_1809_10573_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _clustered(N, seed):
    # rows only in [-N/2, N/8) (the upper leaves are empty); columns avoid [0.25, 0.5)
    rng = np.random.default_rng(seed)
    om = np.sort(rng.uniform(-N / 2, N / 8, N))
    xs = np.sort(np.concatenate([rng.uniform(0.0, 0.25, N // 2), rng.uniform(0.5, 1.0, N - N // 2)]))
    return om, xs


CASES = {
    # name: (points, N, n0 for the depth, eps, build kwargs)
    "nufft_1000": ("random", 1000, 16, 1e-6, {}),
    "nufft_1000_e8": ("random", 1000, 16, 1e-8, {}),
    "nufft_3000_oddL": ("random", 3000, 32, 1e-6, {}),
    "clustered_48_exact": ("clustered", 48, 6, 1e-15, dict(sampler="all")),
    "clustered_640": ("clustered", 640, 10, 1e-8, {}),
}


@functools.lru_cache(maxsize=None)
def case(name):
    kind, N, n0, eps, kw = CASES[name]
    om, xs = inputs.nufft_points(N, seed=N) if kind == "random" else _clustered(N, 5)
    L = idbf.levels_for(N, n0)
    ro, co = idbf.dyadic_leaves(om, -N / 2, N / 2, L), idbf.dyadic_leaves(xs, 0.0, 1.0, L)
    K = kernels.Kernel(kernels.KIND_DFT, sign=-1)
    F = idbf.build(K, om, xs, eps, None, leaves=(ro, co), **kw)
    ex = idbf.export(F)
    return dict(N=N, F=F, ex=ex, om=om, xs=xs, K=K, eps=eps, ro=ro, co=co)


def test_the_cases_have_uneven_and_empty_leaves():
    assert np.diff(case("nufft_1000")["co"]).min() != np.diff(case("nufft_1000")["co"]).max()
    c = case("clustered_640")
    assert np.sum(np.diff(c["ro"]) == 0) >= 2 and np.sum(np.diff(c["co"]) == 0) >= 2
    assert (c["ex"]["seg_len"] == 0).any()
    assert ((c["ex"]["blk_cols"] == 0) & (c["ex"]["blk_rows"] > 0)).any()


MODES = [(P.MODE_FP64, P.STORE_C128, torch.complex128, 1e-12), (P.MODE_DF64, P.STORE_DF64, torch.complex128, 1e-12),
         (P.MODE_FP32, P.STORE_C64, torch.complex64, 2e-5)]


@pytest.mark.parametrize("mode,store,dt,bar", MODES, ids=["fp64", "df64", "fp32"])
@pytest.mark.parametrize("nrhs", [1, 5, 19])
@pytest.mark.parametrize("name", list(CASES))
def test_uneven_leaves_forward_and_adjoint_match_oracle(name, nrhs, mode, store, dt, bar):
    c = case(name)
    plan = P.Plan.import_factors(c["ex"], storage=store)
    st = plan.stats()
    assert st["n0"] == 0 and st["N"] == c["N"]
    X = inputs.complex_gaussian(c["N"], nrhs, seed=31)
    xd = torch.from_numpy(X).to(dt).cuda()
    y = plan.apply(xd, mode=mode).cpu().numpy()
    ya = plan.apply_adjoint(xd, mode=mode).cpu().numpy()
    Xr = xd.cpu().numpy().astype(np.complex128)
    assert rel(y, idbf.apply(c["F"], Xr)) < bar
    assert rel(ya, idbf.apply_adjoint(c["F"], Xr)) < bar


def test_uneven_leaves_against_the_dense_sum():
    # Eq. N of Example 3: u_k = sum_n exp(-2 pi i omega_k x_n) g_n, within 10 eps
    for name in ("nufft_1000", "nufft_3000_oddL"):
        c = case(name)
        plan = P.Plan.import_factors(c["ex"], storage=P.STORE_DF64)
        g = inputs.complex_gaussian(c["N"], 1, seed=2)[:, 0]
        y = plan.apply(torch.from_numpy(g).cuda(), mode=P.MODE_DF64).cpu().numpy()
        assert rel(y, idbf.dense_matvec(c["K"], c["om"], c["xs"], g)) < 10 * c["eps"]


@pytest.mark.parametrize("name", ["nufft_3000_oddL", "clustered_640", "clustered_48_exact"])
@pytest.mark.parametrize("mode,store,dt,bar", MODES[1:], ids=["df64", "fp32"])
def test_uneven_leaves_every_forward_variant(name, mode, store, dt, bar):
    """Uneven and empty leaves through every single-vector forward variant (the streaming kernel
    with its ring layouts and fused level pairs reads leaf offsets and writes zero products for
    blocks without columns; the warp-per-node kernel is refused and falls back), and through the
    autotuner's choice."""
    c = case(name)
    plan = P.Plan.import_factors(c["ex"], storage=store)
    X = inputs.complex_gaussian(c["N"], 1, seed=4)
    xd = torch.from_numpy(X).to(dt).cuda()
    ref = idbf.apply(c["F"], xd.cpu().numpy().astype(np.complex128))
    L = c["ex"]["L"]
    for v in range(P.NUM_FWD_VARIANTS):
        for pat in [[v] * (L + 1)] + ([[1] + [v] * L] if v >= 16 else []):
            plan.set_level_variants(mode, pat)
            y = plan.apply(xd, mode=mode)
            plan.sync_status()
            assert rel(y.cpu().numpy(), ref) < bar, f"variant {v}, pattern {pat}"
    plan.autotune(mode, reps=1)
    assert rel(plan.apply(xd, mode=mode).cpu().numpy(), ref) < bar


def test_uneven_leaves_refuse_the_tensor_cores_and_batches():
    c = case("nufft_1000")
    plan = P.Plan.import_factors(c["ex"], storage=P.STORE_C64)
    with pytest.raises(P.IDBFError):
        plan.apply(torch.zeros((c["N"], 4), dtype=torch.complex64, device="cuda"), mode=P.MODE_TF32X3)
    with pytest.raises(P.IDBFError):
        P.Batch([plan], [1], mode=P.MODE_FP32)


def test_uneven_leaves_allocation_free_apply():
    import ctypes as C
    from paper_1809_10573_gb300 import _lib
    c = case("clustered_640")
    plan = P.Plan.import_factors(c["ex"], storage=P.STORE_C128)
    X = inputs.complex_gaussian(c["N"], 3, seed=5)
    xt = torch.from_numpy(X.T.copy()).cuda()
    yt = torch.full_like(xt, float("nan"))
    st = torch.cuda.current_stream().cuda_stream
    assert _lib.lib().idbf_apply_noalloc(plan._h, C.c_void_p(xt.data_ptr()), C.c_void_p(yt.data_ptr()), 3, c["N"],
                                         P.MODE_FP64, C.c_void_p(st)) == _lib.OK
    torch.cuda.synchronize()
    assert rel(yt.cpu().numpy().T, idbf.apply(c["F"], X)) < 1e-12


@pytest.mark.parametrize("name", ["nufft_1000", "nufft_1000_e8", "nufft_3000_oddL", "clustered_640"])
def test_gpu_built_uneven_leaves_meet_the_tolerance(name):
    """idbf_build_leaves on the coordinate-based trees of the library's own dyadic partition: the
    apply and the adjoint within 10 eps of the dense sum of Eq. N and of K^* (the GPU and the
    oracle constructions are compared through accuracy only: pivot ties may pick different
    skeletons)."""
    c = case(name)
    kind, N, n0, eps, kw = CASES[name]
    L = P.tree_depth(N, n0)
    ro = P.dyadic_leaves(c["om"], -N / 2, N / 2, L)
    co = P.dyadic_leaves(c["xs"], 0.0, 1.0, L)
    assert np.array_equal(ro, c["ro"]) and np.array_equal(co, c["co"])
    plan = P.Plan.build_leaves(c["om"], c["xs"], L, ro, co, eps=eps, kernel="dft", sign=-1,
                               qr_arith=P.QR_DF64 if name == "nufft_1000" else P.QR_FP64)
    st = plan.stats()
    assert st["n0"] == 0 and st["N"] == N and st["rank_saturated"] == 0
    g = inputs.complex_gaussian(N, 2, seed=6)
    Kd = c["K"].entries(c["om"], c["xs"], np.arange(N), np.arange(N))
    y = plan.apply(torch.from_numpy(g).cuda()).cpu().numpy()
    ya = plan.apply_adjoint(torch.from_numpy(g).cuda()).cpu().numpy()
    assert rel(y, Kd @ g) < 10 * eps
    assert rel(ya, Kd.conj().T @ g) < 10 * eps


def test_gpu_built_uneven_leaves_at_a_hundred_thousand_points():
    """N = 100003 random points (Example 3), about 64 per leaf (L = 11): eps^a of Sec. 3 on 256
    rows against the direct sum computed on the GPU, within 10 eps."""
    N, n0, eps = 100003, 64, 1e-6
    om, xs = inputs.nufft_points(N, seed=17)
    L = P.tree_depth(N, n0)
    ro, co = P.dyadic_leaves(om, -N / 2, N / 2, L), P.dyadic_leaves(xs, 0.0, 1.0, L)
    plan = P.Plan.build_leaves(om, xs, L, ro, co, eps=eps, kernel="dft", sign=-1)
    g = torch.from_numpy(inputs.complex_gaussian(N, 1, seed=2)[:, 0]).cuda()
    y = plan.apply(g)
    rows = torch.from_numpy(inputs.sample_rows(N, 256, seed=3)).cuda()
    ud = P.kernel_matvec_rows(torch.from_numpy(om).cuda(), torch.from_numpy(xs).cuda(), g, rows, kernel="dft", sign=-1)
    assert float(torch.linalg.norm(y[rows] - ud) / torch.linalg.norm(ud)) < 10 * eps
