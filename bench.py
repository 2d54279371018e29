#!/usr/bin/env python3
"""Throughput of the IDBF apply: applies/s at N = 2^20 on one GB300 (replicas on N GPUs).

Workload (the configuration the headline metric is quoted on): the 1D FIO
K(x, xi) = exp(2 pi i (x xi + c(x) |xi|)), c(x) = (2 + sin 2 pi x sin 4 pi x) / 3, on the uniform
grids x_i = i/N, xi_j = j - N/2, N = 2^20, eps = 1e-6, leaf n0 = 64, one complex128 right-hand
side drawn from a seeded complex Gaussian. The factorization is built on the GPU (untimed);
a step is one apply y = K x through all L + 1 = 15 butterfly levels.

Modes timed: "df64" (factors as double-float pairs, FP32-pair arithmetic, FP64-class accuracy;
the headline value), "fp64" (FP64 factors and FMA), "fp32" (complex64 factors and FP32 FMA).
Each states its relative error against the FP64 apply, and the FP64 apply states eps^a of
Sec. 3 against dense rows of K x computed directly on the GPU.

`--impl reference` times the CPU oracle instead (see cpu_arm below); there is no other
implementation to compare with.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")  # the oracle runs single-threaded (the paper's setting)

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_LOG2 = 20     # default; --log2n changes it (smaller cases for profiling)
LEAF = 64
EPS = 1e-6
T_OVERSAMPLE, T_LEAF = 2.0, 4.0
SEED = 2
CPU_LOG2 = 14   # the bounded CPU sample: the same workload at N = 2^14
METRIC = "IDBF applies/s at N=2^20 (FP64 vs split-FP32, rel err stated), % HBM roofline"


def workload(log2n):
    return (f"1D FIO c(x)=(2+sin2pi x sin4pi x)/3, X={{i/N}}, Omega={{j-N/2}}, N=2^{log2n}, eps=1e-6, leaf 64, "
            "Mock-Chebyshev t=2 (t=4 at the leaf), complex128, 1 RHS (seeded complex Gaussian)")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def fp32_fma_peak():
    """FP32 FMA peak of the GPU in TFMA/s from its unit counts and clock: SMs x 128 FP32 lanes
    (one FMA per lane per cycle) x the maximum SM clock (MEASURED_PEAKS.json, else the device)."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f)["sm_max_mhz"])
    except Exception:
        pass
    if mhz is None:
        mhz = 2070.0
    return sms * 128 * mhz * 1e6 / 1e12, f"{sms} SMs x 128 FP32 FMA/clk x {mhz:.0f} MHz"


def parse_level_variants(spec):
    """'df64=7,1,10;fp32=7,3,1' -> {'df64': [7, 1, 10], 'fp32': [7, 3, 1]}."""
    out = {}
    for part in (spec or "").split(";"):
        if part.strip():
            name, vals = part.split("=", 1)
            out[name.strip()] = [int(v) for v in vals.split(",")]
    return out


def code_digest(src: str) -> str:
    """sha256 of C/CUDA source with its comments, trailing blanks and blank lines removed: an
    edit of comments leaves the code, and so the profiled DRAM traffic, unchanged."""
    import hashlib
    import re
    s = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    s = re.sub(r"//[^\n]*", "", s)
    lines = [ln.rstrip() for ln in s.splitlines()]
    return hashlib.sha256("\n".join(ln for ln in lines if ln).encode()).hexdigest()


def read_traffic_summary():
    """DRAM bytes per algorithmic byte of the level kernel from the committed ncu summary, valid
    only while the kernel's code is the one that was profiled (code_digest of apply.cu)."""
    path = os.path.join(ROOT, "profiles", "level_kernel_traffic.txt")
    try:
        kv = {}
        for ln in open(path):
            if "=" in ln and not ln.startswith("#"):
                k, v = ln.strip().split("=", 1)
                kv[k.strip()] = v.strip()
        src = open(os.path.join(ROOT, "paper_1809_10573_gb300", "csrc", "apply.cu"), encoding="utf-8").read()
        if code_digest(src) != kv.get("apply_cu_code_sha256"):
            return None
        return float(kv["dram_bytes_per_algorithmic_byte"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while active."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = None

    def __enter__(self):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            self.f.flush()
            self.f.seek(0)
            for ln in self.f.read().splitlines():
                p = [x.strip() for x in ln.split(",")]
                if len(p) >= 10:
                    rows.append(p)
            os.unlink(self.f.name)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[4]) for r in rows if r[4].replace(".", "").isdigit()) if rows else None}


def dist_init():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend, init_method="env://")
    elif torch.cuda.is_available():
        torch.cuda.set_device(local)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(value: float, world: int) -> float:
    """The slowest rank's time decides the job's time."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, seconds_per_rank: float, world: int) -> tuple:
    """Whole-job throughput: every rank's units over the slowest rank's time (weak scaling)."""
    t = max_over_ranks(seconds_per_rank, world)
    return units_per_rank * world / t, t


# ---- CPU oracle (the baseline; the only place bench.py runs oracle/) ------------------------
def oracle_sample():
    """The oracle's factorization of the same workload at N = 2^14 (build untimed)."""
    from oracle import idbf, kernels
    from paper_1809_10573_gb300 import inputs
    N = 1 << CPU_LOG2
    x, xi = inputs.uniform_grid(N)
    F = idbf.build(kernels.Kernel(kernels.KIND_FIO, c_profile=0), x, xi, EPS, LEAF, t=T_OVERSAMPLE, t_leaf=T_LEAF)
    g = inputs.complex_gaussian(N, 1, seed=SEED)[:, 0]
    return F, g


def nlogn_scale():
    """Work of one N = 2^log2n apply over one N = 2^14 apply, O(N log N) (Sec. 1)."""
    return ((1 << N_LOG2) * N_LOG2) / ((1 << CPU_LOG2) * CPU_LOG2)


def cpu_time_applies(F, g, reps=None, budget_s=10.0):
    from oracle import idbf
    idbf.apply(F, g)
    times = []
    t_end = time.perf_counter() + budget_s
    while (reps is None and time.perf_counter() < t_end) or (reps is not None and len(times) < reps):
        t0 = time.perf_counter()
        idbf.apply(F, g)
        times.append(time.perf_counter() - t0)
    return times


def cpu_baseline():
    F, g = oracle_sample()
    times = cpu_time_applies(F, g)
    t = statistics.median(times)
    return {"value": 1.0 / (t * nlogn_scale()), "unit": "applies/s", "cores": 1, "kind": "oracle",
            "sample": (f"oracle FP64 apply (numpy, 1 thread) of the same workload at N=2^{CPU_LOG2} "
                       f"(factors built by the oracle, untimed), median of {len(times)} applies = {t*1e3:.1f} ms, "
                       f"scaled to one N=2^{N_LOG2} apply by the N log N work ratio {nlogn_scale():.1f}")}


def cpu_arm(args, rank, world):
    if rank != 0:
        return 0
    F, g = oracle_sample()
    cpu_time_applies(F, g, reps=args.warmup)
    t0 = time.perf_counter()
    cpu_time_applies(F, g, reps=args.steps)
    dt = time.perf_counter() - t0
    per = dt / args.steps
    value = 1.0 / (per * nlogn_scale())
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "applies/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3 * nlogn_scale(),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload(N_LOG2)},
            "cpu_baseline": {"value": value, "unit": "applies/s", "cores": 1, "kind": "oracle",
                             "sample": (f"each step: one oracle FP64 apply at N=2^{CPU_LOG2} of the same workload "
                                        f"({per*1e3:.1f} ms), scaled by the N log N work ratio {nlogn_scale():.1f}")},
            "e2e": {"value": value, "unit": "applies/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---- GPU arm ---------------------------------------------------------------------------------
def gpu_arm(args, rank, world, local):
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_1809_10573_gb300 as P
    from paper_1809_10573_gb300 import inputs

    N = 1 << N_LOG2
    x, xi = inputs.uniform_grid(N)
    t0 = time.time()
    plan = P.Plan.build(x, xi, eps=EPS, leaf=LEAF, kernel="fio", c_profile=0, oversample=T_OVERSAMPLE,
                        oversample_leaf=T_LEAF)
    build_s = time.time() - t0
    want = set(args.modes.split(","))
    fmts = [f for name, f in (("fp64", P.STORE_C128), ("df64", P.STORE_DF64), ("fp32", P.STORE_C64)) if name in want]
    if "df64" not in want:
        raise SystemExit("the headline mode df64 must be among --modes")
    if "fp64" not in want:   # the FP64 reference result is computed before the C128 copy goes
        fmts_final = fmts
        fmts = sorted(set(fmts) | {P.STORE_C128})
    else:
        fmts_final = fmts
    plan.set_storage(*fmts)
    st = plan.stats()
    L = st["L"]
    g = inputs.complex_gaussian(N, 1, seed=SEED)[:, 0]
    gd = torch.from_numpy(g).cuda()
    g32 = gd.to(torch.complex64)
    stream = torch.cuda.current_stream()

    # accuracy: eps^a of the FP64 apply on 256 sampled rows against the direct matvec (Sec. 3),
    # and each mode against the FP64 apply
    y64 = plan.apply(gd, mode=P.MODE_FP64)
    rows = inputs.sample_rows(N, 256, seed=SEED)
    ud = P.kernel_matvec_rows(torch.from_numpy(x).cuda(), torch.from_numpy(xi).cuda(), gd,
                              torch.from_numpy(rows).cuda(), kernel="fio", c_profile=0)
    eps_a = float(torch.linalg.norm(y64[torch.from_numpy(rows).cuda()] - ud) / torch.linalg.norm(ud))
    ydf = plan.apply(gd, mode=P.MODE_DF64)
    y32 = plan.apply(g32, mode=P.MODE_FP32) if "fp32" in want else None
    nrm = torch.linalg.norm(y64)
    rel_df = float(torch.linalg.norm(ydf - y64) / nrm)
    rel_32 = float(torch.linalg.norm(y32.to(torch.complex128) - y64) / nrm) if "fp32" in want else None
    plan.set_storage(*fmts_final)

    # autotuner: fastest forward kernel per level for each timed mode (untimed), unless the
    # variants are given (e.g. to profile exactly the choices of an earlier uninstrumented run)
    tune = {}
    fixed = parse_level_variants(args.level_variants)
    for name, mode in (("df64", P.MODE_DF64), ("fp32", P.MODE_FP32)):
        if name in want:
            fmt = P.STORE_DF64 if name == "df64" else P.STORE_C64
            if name in fixed:
                if len(fixed[name]) != L + 1:
                    raise SystemExit(f"--level-variants {name}: {L + 1} values expected")
                plan.set_level_variants(mode, fixed[name])
                tune[name] = {"level_variants": plan.stats()["level_variant"][fmt], "given": True}
                continue
            ms_sum = plan.autotune(mode, reps=10)  # short levels run for ~30 us: enough launches to rank them
            tune[name] = {"level_variants": plan.stats()["level_variant"][fmt], "sum_of_level_ms": ms_sum}

    def timed(mode, vec, steps, warmup, sampler_index=None):
        for _ in range(warmup):
            plan.apply(vec, mode=mode, out=ybuf[mode])
        barrier(world)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            plan.apply(vec, mode=mode, out=ybuf[mode])
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        return e0.elapsed_time(e1) / 1e3

    ybuf = {P.MODE_FP64: torch.empty_like(gd), P.MODE_DF64: torch.empty_like(gd), P.MODE_FP32: torch.empty_like(g32)}
    modes = {}
    for name, mode, vec, eb in (("fp64", P.MODE_FP64, gd, 16), ("fp32", P.MODE_FP32, g32, 8)):
        if name not in want:
            continue
        secs = timed(mode, vec, max(5, args.steps // 2), args.warmup)
        n = max(5, args.steps // 2)
        ab = plan.algorithmic_bytes(1, eb, eb)
        modes[name] = {"applies_per_s": n / secs, "ms_per_apply": secs / n * 1e3,
                       "algorithmic_GBps": ab * n / secs / 1e9,
                       "rel_err_vs_fp64": 0.0 if name == "fp64" else rel_32}
        if name == "fp64":
            # the FP64 apply is bound by the FP64 FMA pipes: 4 DFMA per stored complex entry
            sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
            dpk = sms * 2 * 2070e6 / 1e12  # 2 FP64 FMA per SM per clock (1.25 TFLOP/s nominal) x max clock
            dfma = 4.0 * plan.stats()["entries"] * n / secs / 1e12
            modes[name]["alu"] = {"achieved_TDFMA_per_s": dfma, "peak_TDFMA_per_s": dpk, "frac": dfma / dpk,
                                  "peak_kind": f"derived: {sms} SMs x 2 FP64 FMA/clk x 2070 MHz"}
    # headline: double-float, clocks sampled during the timed region
    with ClockSampler(torch.cuda.current_device()) as cs:
        secs = timed(P.MODE_DF64, gd, args.steps, args.warmup)
    clocks = cs.summary()
    value, tmax = job_throughput(args.steps, secs, world)
    ms = tmax / args.steps * 1e3
    ab = plan.algorithmic_bytes(1, 16, 16)
    modes["df64"] = {"applies_per_s": args.steps / secs, "ms_per_apply": secs / args.steps * 1e3,
                     "algorithmic_GBps": ab * args.steps / secs / 1e9, "rel_err_vs_fp64": rel_df}
    peak, peak_kind = peaks()
    achieved = ab / (secs / args.steps) / 1e9   # all L+1 launches are the level kernel
    ratio = read_traffic_summary()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_kind": peak_kind,
                "traffic": (ratio * ab / (L + 1)) if ratio is not None else None,
                "kernel": "double-float level kernels (per level the autotuned k_level_stream ring or "
                          "k_level_fwd; every launch of the timed region is one of them)",
                "algorithmic_bytes_per_launch": ab / (L + 1)}
    # end to end through the C call: pinned host x -> device, apply, device -> host y
    xh = torch.from_numpy(g.copy()).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    xdev = torch.empty_like(gd)
    ydev = torch.empty_like(gd)

    def e2e_step():
        xdev.copy_(xh, non_blocking=True)
        plan.apply(xdev, mode=P.MODE_DF64, out=ydev)
        yh.copy_(ydev, non_blocking=True)

    for _ in range(args.warmup):
        e2e_step()
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_secs = e0.elapsed_time(e1) / 1e3
    e2e_value, _ = job_throughput(args.steps, e2e_secs, world)
    if not torch.allclose(yh.cuda(), ydf):
        raise RuntimeError("end-to-end result differs from the device apply")
    cpu = cpu_baseline() if (rank == 0 and world == 1 and not args.no_cpu) else None
    line = {"metric": METRIC, "value": value, "unit": "applies/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32x2", "data": "synthetic",
            "config": {"workload": workload(N_LOG2), "N": N, "eps": EPS, "leaf": LEAF, "nrhs": 1,
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                       "l2": f"inputs larger than L2: {st['entries']*16/1e9:.1f} GB of factors per apply"},
            "rel_err": {"eps_a_fp64_vs_dense_256_rows": eps_a, "df64_vs_fp64": rel_df, "fp32_vs_fp64": rel_32},
            "roofline": roofline, "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "applies/s", "h2d_bytes_per_step": N * 16, "d2h_bytes_per_step": N * 16},
            "gpu_launches": (L + 1) * args.steps, "clocks": clocks, "modes": modes, "autotune": tune,
            "build": {"seconds": build_s, "entries": st["entries"], "levels": L + 1,
                      "level_kmax": st["level_kmax"], "level_entries": st["level_entries"],
                      "rank_saturated": st["rank_saturated"],
                      "device_GB": st["device_bytes"] / 1e9}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


# ---- further workloads (separate JSON lines; the default run is the single-vector apply) ------
def gpu_mrhs(args, rank, world):
    """Many right-hand sides: N = 2^18, eps = 1e-6, 256 RHS; complex FP32 factors with 3xTF32
    tensor-core block products vs the FP64 apply of the same vectors on the same GPU."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_1809_10573_gb300 as P
    from paper_1809_10573_gb300 import inputs
    N, R = 1 << (args.log2n if args.log2n is not None else 18), 256
    x, xi = inputs.uniform_grid(N)
    plan = P.Plan.build(x, xi, eps=EPS, leaf=LEAF, kernel="fio", c_profile=0, oversample=T_OVERSAMPLE,
                        oversample_leaf=T_LEAF)
    plan.set_storage(P.STORE_C128, P.STORE_C64)
    X = torch.from_numpy(inputs.complex_gaussian(N, R, seed=3)).cuda()
    X32 = X.to(torch.complex64)

    def tm(mode, xx, steps):
        for _ in range(args.warmup):
            plan.apply(xx, mode=mode)
        barrier(world)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            y = plan.apply(xx, mode=mode)
        e1.record()
        torch.cuda.synchronize()
        return y, e0.elapsed_time(e1) / 1e3 / steps

    ytc, stc = tm(P.MODE_TF32X3, X32, args.steps)
    plan.sync_status()
    y64, s64 = tm(P.MODE_FP64, X, 1)
    err = float(torch.linalg.norm(ytc.to(torch.complex128) - y64) / torch.linalg.norm(y64))
    st = plan.stats()
    flops = 24.0 * st["entries"] * R  # 8 real flops per complex entry and rhs, three split products
    value, tmax = job_throughput(1.0, stc, world)
    lg = N.bit_length() - 1
    line = {"metric": f"IDBF multi-RHS applies/s at N=2^{lg}, 256 RHS (3xTF32 tensor cores, error vs FP64 stated)",
            "value": value, "unit": "applies/s (256 rhs each)", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tmax * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "tf32x3", "data": "synthetic",
            "config": {"workload": f"1D FIO N=2^{lg} eps=1e-6 leaf 64, 256 complex Gaussian RHS (seed 3), complex64 factors"},
            "rel_err_vs_fp64": err, "vector_applies_per_s": value * R,
            "roofline": {"bound": "tensor", "achieved": flops / stc / 1e12, "unit": "TFLOP/s",
                         "peak": 1939.7 / 2, "peak_kind": "measured bf16 burst x 1/2 (nominal tf32:bf16 ratio)",
                         "frac": flops / stc / 1e12 / (1939.7 / 2)},
            "fp64_same_rhs": {"ms_per_apply": s64 * 1e3, "speedup_tf32x3_vs_fp64": s64 / stc}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def gpu_batch(args, rank, world):
    """Uneven batch: 64 operators, N = 2^e with e uniform in [12, 18], the first half the FIO and
    the second half the jittered DFT kernel, 1-32 RHS each, eps = 1e-6, one persistent launch in a
    CUDA graph, tiles autotuned. Timed in FP32 (the line's value) and in double-float, each beside
    the same 64 applies made one plan at a time; errors against the FP64 apply."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_1809_10573_gb300 as P
    from paper_1809_10573_gb300 import inputs
    ops = inputs.uneven_batch(seed=4)
    if args.log2n is not None:  # a smaller batch for profiling: the same draw, N capped at 2^log2n
        ops = [dict(o, N=min(o["N"], 1 << args.log2n)) for o in ops]
    plans, xs = [], []
    t0 = time.time()
    for o in ops:
        N = o["N"]
        if o["kind"] == "fio":
            x, xi = inputs.uniform_grid(N)
            p = P.Plan.build(x, xi, eps=EPS, leaf=LEAF, kernel="fio", c_profile=0, oversample=T_OVERSAMPLE,
                             oversample_leaf=T_LEAF)
        else:
            x, xi = inputs.jittered_grid(N, seed=o["seed"])
            p = P.Plan.build(x, xi, eps=EPS, leaf=LEAF, kernel="dft", sign=-1)
        plans.append(p)
        xs.append(torch.from_numpy(inputs.complex_gaussian(N, o["nrhs"], seed=o["seed"])).cuda())
    build_s = time.time() - t0
    y64 = [p.apply(x, mode=P.MODE_FP64) for p, x in zip(plans, xs)]

    def timed(fn, steps):
        for _ in range(args.warmup):
            fn()
        barrier(world)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / steps

    res = {}
    # the factors of all 64 operators take ~190 GB per 16-byte format: convert in place, one
    # format at a time (C128 -> double-float -> complex64)
    for name, mode, store, vdt, eb in (("df64", P.MODE_DF64, P.STORE_DF64, torch.complex128, 16),
                                       ("fp32", P.MODE_FP32, P.STORE_C64, torch.complex64, 8)):
        for p in plans:
            p.set_storage(store)
        torch.cuda.synchronize()
        xm = [x.to(vdt) for x in xs]
        ym = [torch.empty_like(x) for x in xm]
        b = P.Batch(plans, [o["nrhs"] for o in ops], mode=mode)
        tuned_ms = b.autotune(xm, reps=2)
        secs = timed(lambda: b.apply(xm, ym), args.steps)
        b.sync_status()
        err = max(float(torch.linalg.norm(y.to(torch.complex128) - r) / torch.linalg.norm(r)) for y, r in zip(ym, y64))
        sep = timed(lambda: [p.apply(x, mode=mode) for p, x in zip(plans, xm)], max(1, args.steps // 4))
        algo = sum(p.algorithmic_bytes(x.shape[1], eb, eb) for p, x in zip(plans, xs))
        fma = sum(4.0 * p.stats()["entries"] * x.shape[1] for p, x in zip(plans, xs))  # real FMA per complex MAC: 4
        res[name] = {"ms_per_batch": secs * 1e3, "batches_per_s": 1.0 / secs, "algorithmic_GBps": algo / secs / 1e9,
                     "useful_TFMA_per_s": fma / secs / 1e12,
                     "algorithmic_bytes": algo, "max_rel_err_vs_fp64": err, "tiles": b.info(),
                     "autotune_best_ms": tuned_ms, "separate_applies_ms": sep * 1e3,
                     "speedup_vs_separate_applies": sep / secs}
        b.close()
    value, tmax = job_throughput(1.0, res["fp32"]["ms_per_batch"] / 1e3, world)
    peak, kind = peaks()
    fpk, fpk_how = fp32_fma_peak()
    r32 = res["fp32"]
    line = {"metric": "IDBF uneven-batch applies/s (64 operators, N 2^12..2^18, 1-32 RHS, one persistent launch in a CUDA graph)",
            "value": value, "unit": "batches/s (64 operator applies each)", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tmax * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "64 ops, seed 4: FIO (ops 0-31) / jittered DFT (32-63), eps=1e-6, leaf 64, complex64 factors"
                                   + (f", N capped at 2^{args.log2n}" if args.log2n is not None else "")},
            "rel_err": {"max_over_ops_vs_fp64": r32["max_rel_err_vs_fp64"]},
            "operator_applies_per_s": 64 * value, "vector_applies_per_s": sum(o["nrhs"] for o in ops) * value,
            # 1-32 right-hand sides make ~8 FMA per factor byte: the FP32 FMA pipes, not HBM, bound it
            "roofline": {"bound": "alu", "achieved": r32["useful_TFMA_per_s"], "peak": fpk, "unit": "TFMA/s",
                         "frac": r32["useful_TFMA_per_s"] / fpk, "peak_kind": "derived: " + fpk_how,
                         "hbm_GBps": r32["algorithmic_GBps"], "hbm_frac_of_measured": r32["algorithmic_GBps"] / peak},
            "modes": res, "build_seconds_total": build_s, "N": [o["N"] for o in ops], "nrhs": [o["nrhs"] for o in ops]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def gpu_autograd(args, rank, world):
    """Differentiation: loss ||K x - b||^2 at N = 2^20, eps = 1e-6, complex FP32, 32 RHS; forward
    apply and hand-written adjoint backward through torch.autograd."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_1809_10573_gb300 as P
    from paper_1809_10573_gb300 import inputs
    N, R = 1 << (args.log2n if args.log2n is not None else 20), 32
    x, xi = inputs.uniform_grid(N)
    plan = P.Plan.build(x, xi, eps=EPS, leaf=LEAF, kernel="fio", c_profile=0, oversample=T_OVERSAMPLE,
                        oversample_leaf=T_LEAF)
    plan.set_storage(P.STORE_C64)
    X = torch.from_numpy(inputs.complex_gaussian(N, R, seed=5)).to(torch.complex64).cuda()
    B = torch.from_numpy(inputs.complex_gaussian(N, R, seed=6)).to(torch.complex64).cuda()

    def step():
        xv = X.clone().requires_grad_(True)
        loss = ((P.apply(plan, xv, P.MODE_FP32) - B).abs() ** 2).sum()
        loss.backward()
        return loss, xv.grad

    for _ in range(args.warmup):
        step()
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        loss, g = step()
    e1.record()
    torch.cuda.synchronize()
    secs = e0.elapsed_time(e1) / 1e3 / args.steps
    value, tmax = job_throughput(1.0, secs, world)
    fpk, fpk_how = fp32_fma_peak()
    lg = N.bit_length() - 1
    line = {"metric": f"IDBF forward+backward steps/s at N=2^{lg}, 32 RHS (loss ||Kx-b||^2, adjoint-butterfly backward)",
            "value": value, "unit": "fwd+bwd/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tmax * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"1D FIO N=2^{lg} eps=1e-6 leaf 64, 32 RHS complex64 (x seed 5, b seed 6)"},
            "loss": float(loss.detach()), "grad_norm": float(torch.linalg.norm(g)),
            # forward and adjoint: 4 real FMA per stored complex entry and right-hand side each
            "roofline": {"bound": "alu", "achieved": 8.0 * plan.stats()["entries"] * R / secs / 1e12,
                         "peak": fpk, "unit": "TFMA/s", "frac": 8.0 * plan.stats()["entries"] * R / secs / 1e12 / fpk,
                         "peak_kind": "derived: " + fpk_how}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--log2n", type=int, default=None,
                    help="N = 2^log2n (default: the benchmarked size of the workload, 20 for apply and "
                         "autograd, 18 for mrhs; smaller cases for profiling)")
    ap.add_argument("--modes", default="df64,fp64,fp32", help="apply modes to time (df64 is the headline)")
    ap.add_argument("--level-variants", default=None,
                    help="per-level forward variants instead of the autotuner, e.g. 'df64=7,1,10,...;fp32=...' "
                         "(apply workload)")
    ap.add_argument("--workload", choices=["apply", "mrhs", "batch", "autograd"], default="apply",
                    help="apply: the headline single-vector apply at N=2^20; the others print their own lines")
    args = ap.parse_args()
    global N_LOG2
    N_LOG2 = args.log2n if args.log2n is not None else 20
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")
    rank, world, local = dist_init()
    try:
        if args.impl == "reference":
            return cpu_arm(args, rank, world)
        if args.workload == "mrhs":
            return gpu_mrhs(args, rank, world)
        if args.workload == "batch":
            return gpu_batch(args, rank, world)
        if args.workload == "autograd":
            return gpu_autograd(args, rank, world)
        return gpu_arm(args, rank, world, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
