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


def parse_level_variants(spec):
    """'df64=7,1,10;fp32=7,3,1' -> {'df64': [7, 1, 10], 'fp32': [7, 3, 1]}."""
    out = {}
    for part in (spec or "").split(";"):
        if part.strip():
            name, vals = part.split("=", 1)
            out[name.strip()] = [int(v) for v in vals.split(",")]
    return out


def launches_per_apply(variants, L):
    """Level-kernel launches of one single-vector forward apply: a fused-pair variant (16-19) on
    level l < L runs levels l and l + 1 in one launch."""
    n, l = 0, 0
    while l <= L:
        v = variants[l] if l < len(variants) else -1
        l += 2 if 16 <= v <= 19 and l < L else 1
        n += 1
    return n


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
# The oracle's FP64 apply costs a fixed time per stored factor entry (measured on the GB300 host
# at N = 2^12 .. 2^15 of this workload: 2.02-2.17 ns per entry on one core), so a bounded sample,
# the same workload at N = 2^14 built by the oracle itself, is scaled to one N = 2^20 apply by the
# ratio of stored entries. Workers are separate processes started with "spawn" (no CUDA state is
# inherited), one per host core, each applying its own copy of the factorization.
E20_STORED_ENTRIES = 3395558732  # stored entries of the N = 2^20 factorization (idbf_stats of the build)


def _oracle_worker(wid, log2n, start, done, ready, results, steps_single, steps_all):
    import os as _os
    for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        _os.environ[_v] = "1"
    sys.path.insert(0, ROOT)
    from oracle import idbf, kernels
    from paper_1809_10573_gb300 import inputs
    N = 1 << log2n
    x, xi = inputs.uniform_grid(N)
    F = idbf.build(kernels.Kernel(kernels.KIND_FIO, c_profile=0), x, xi, EPS, LEAF, t=T_OVERSAMPLE, t_leaf=T_LEAF)
    g = inputs.complex_gaussian(N, 1, seed=SEED)[:, 0]
    entries = sum(s["entries"] for s in idbf.stats(F))
    idbf.apply(F, g)
    ready.put((wid, entries))
    # phase 1: worker 0 alone (one core); phase 2: every worker at once (all cores). Each step is
    # bracketed by the two barriers, so that the parent times the slowest worker of the step.
    for phase, steps in ((0, steps_single), (1, steps_all)):
        for _ in range(steps):
            start.wait(timeout=600)
            if phase == 1 or wid == 0:
                idbf.apply(F, g)
            done.wait(timeout=600)
    results.put(wid)


class OracleTeam:
    """`workers` spawned processes, each building the oracle's factorization at N = 2^log2n on
    construction (in the background) and applying it in timed steps on request."""

    def __init__(self, workers, log2n, steps_single, steps_all):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        self.W, self.log2n = workers, log2n
        self.steps_single, self.steps_all = steps_single, steps_all
        self.start, self.done = ctx.Barrier(workers + 1), ctx.Barrier(workers + 1)
        self.ready, self.results = ctx.Queue(), ctx.Queue()
        self.procs = [ctx.Process(target=_oracle_worker, args=(w, log2n, self.start, self.done, self.ready,
                                                               self.results, steps_single, steps_all), daemon=True)
                      for w in range(workers)]
        for p in self.procs:
            p.start()
        self.entries = None

    def wait_ready(self, timeout=900):
        got = [self.ready.get(timeout=timeout) for _ in range(self.W)]
        self.entries = got[0][1]

    def run(self):
        """Wall time of every step of both phases (seconds)."""
        if self.entries is None:
            self.wait_ready()
        times = []
        for steps in (self.steps_single, self.steps_all):
            ts = []
            for _ in range(steps):
                self.start.wait(timeout=600)
                t0 = time.perf_counter()
                self.done.wait(timeout=600)
                ts.append(time.perf_counter() - t0)
            times.append(ts)
        for _ in range(self.W):
            self.results.get(timeout=600)
        for p in self.procs:
            p.join(timeout=60)
        return times

    def close(self):
        for p in self.procs:
            if p.is_alive():
                p.terminate()


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_summary(team, times, e20):
    """cpu_baseline object from the two phases of an OracleTeam run."""
    single, allc = times
    scale = e20 / team.entries
    t1 = statistics.median(single)
    tw = statistics.median(allc)
    one = 1.0 / (t1 * scale)
    allv = team.W / (tw * scale)
    return {"value": allv, "unit": "applies/s", "cores": team.W, "kind": "oracle",
            "sample": (f"oracle FP64 apply (numpy, one thread per process) of the same workload at N=2^{team.log2n} "
                       f"(built by the oracle, untimed; {team.entries} stored entries): {team.W} processes each "
                       f"applying its own copy at once, median step {tw*1e3:.1f} ms over {len(allc)} steps; scaled to one "
                       f"N=2^20 apply by the ratio of stored entries {e20}/{team.entries} = {scale:.1f} (the oracle "
                       f"apply costs a fixed time per stored entry: 2.02-2.17 ns/entry on one Grace core at N=2^12..2^15)"),
            "single_core": {"value": one, "unit": "applies/s", "cores": 1,
                            "ms_per_sample_apply": t1 * 1e3, "ns_per_stored_entry": t1 / team.entries * 1e9,
                            "steps": len(single)},
            "all_cores_ms_per_step": tw * 1e3, "ns_per_stored_entry_all_cores": tw / team.entries / team.W * 1e9}


def cpu_arm(args, rank, world):
    """The reference arm: the CPU oracle (the paper publishes no code) timed on the host cores."""
    if rank != 0:
        return 0
    W = host_cores()
    team = OracleTeam(W, CPU_LOG2, steps_single=args.warmup, steps_all=args.warmup + args.steps)
    try:
        times = team.run()
    finally:
        team.close()
    warm_all = times[1][:args.warmup]
    timed = times[1][args.warmup:]
    per = sum(timed) / len(timed)
    scale = E20_STORED_ENTRIES / team.entries
    value = W / (per * scale)
    cb = cpu_summary(team, [times[0], timed], E20_STORED_ENTRIES)
    del warm_all
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "applies/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload(N_LOG2),
                                            "sample_per_step": f"{W} oracle applies at N=2^{CPU_LOG2} at once "
                                                               f"(one per host core), entry-scaled to N=2^20"},
            "cpu_baseline": dict(cb, value=value),
            "e2e": {"value": value, "unit": "applies/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---- GPU arm ---------------------------------------------------------------------------------
def library_peaks():
    """Arithmetic peaks of this GPU measured in this run by library GEMMs (cuBLAS through torch,
    8192^3, best of a few, CUDA events): FP64, FP32 (TF32 off) and TF32 tensor cores. They are the
    denominators of the ALU / tensor roofline fractions below; no GPU setting is changed."""
    import torch

    def tflops(dtype, tf32, reps):
        prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = tf32
        try:
            n = 8192
            a = torch.randn(n, n, device="cuda", dtype=dtype)
            b = torch.randn(n, n, device="cuda", dtype=dtype)
            for _ in range(2):
                a @ b
            torch.cuda.synchronize()
            best = float("inf")
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                a @ b
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1) / 1e3)
            del a, b
            return 2.0 * n ** 3 / best / 1e12
        finally:
            torch.backends.cuda.matmul.allow_tf32 = prev

    out = {"fp64_tflops": tflops(torch.float64, False, 3), "fp32_tflops": tflops(torch.float32, False, 5),
           "tf32_tflops": tflops(torch.float32, True, 5),
           "how": "cuBLAS GEMM 8192^3 via torch.matmul in this run, best of 3-5 (CUDA events)"}
    torch.cuda.empty_cache()
    return out


def timed_loop(fn, steps, warmup, world, stream=None):
    """Seconds per call of fn over `steps` calls after `warmup`, CUDA events on the stream."""
    import torch
    for _ in range(warmup):
        fn()
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    return e0.elapsed_time(e1) / 1e3 / steps


def gpu_arm(args, rank, world, local):
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_1809_10573_gb300 as P
    from paper_1809_10573_gb300 import inputs

    # the CPU baseline's workers build the oracle's factorizations meanwhile (spawned processes)
    team = None
    if rank == 0 and world == 1 and not args.no_cpu:
        team = OracleTeam(host_cores(), CPU_LOG2, steps_single=5, steps_all=10)
    try:
        line = _gpu_headline(args, rank, world, np, torch, P, inputs, team)
    finally:
        if team is not None:
            team.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def _gpu_headline(args, rank, world, np, torch, P, inputs, team):
    lpk = library_peaks()
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

    ybuf = {P.MODE_FP64: torch.empty_like(gd), P.MODE_DF64: torch.empty_like(gd), P.MODE_FP32: torch.empty_like(g32)}
    modes = {}
    for name, mode, vec, eb in (("fp64", P.MODE_FP64, gd, 16), ("fp32", P.MODE_FP32, g32, 8)):
        if name not in want:
            continue
        n = max(5, args.steps // 2)
        sec = timed_loop(lambda: plan.apply(vec, mode=mode, out=ybuf[mode]), n, args.warmup, world, stream)
        ab = plan.algorithmic_bytes(1, eb, eb)
        modes[name] = {"applies_per_s": 1.0 / sec, "ms_per_apply": sec * 1e3,
                       "algorithmic_GBps": ab / sec / 1e9,
                       "rel_err_vs_fp64": 0.0 if name == "fp64" else rel_32}
        if name == "fp64":
            # the FP64 apply is bound by the FP64 pipes: 4 DFMA (8 flops) per stored complex entry
            tfl = 8.0 * plan.stats()["entries"] / sec / 1e12
            modes[name]["alu"] = {"achieved_TFLOPs": tfl, "peak_TFLOPs": lpk["fp64_tflops"],
                                  "frac": tfl / lpk["fp64_tflops"],
                                  "peak_kind": "measured in this run: cuBLAS DGEMM 8192^3"}
    # headline: double-float, clocks sampled during the timed region
    with ClockSampler(torch.cuda.current_device()) as cs:
        sec = timed_loop(lambda: plan.apply(gd, mode=P.MODE_DF64, out=ybuf[P.MODE_DF64]), args.steps, args.warmup,
                         world, stream)
    clocks = cs.summary()
    value, tmax = job_throughput(1.0, sec, world)
    ms = tmax * 1e3
    ab = plan.algorithmic_bytes(1, 16, 16)
    modes["df64"] = {"applies_per_s": 1.0 / sec, "ms_per_apply": sec * 1e3,
                     "algorithmic_GBps": ab / sec / 1e9, "rel_err_vs_fp64": rel_df}
    peak, peak_kind = peaks()
    achieved = ab / sec / 1e9   # every launch of the timed region is a level kernel
    nlaunch = launches_per_apply(plan.stats()["level_variant"][P.STORE_DF64], L)
    ratio = read_traffic_summary()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_kind": peak_kind,
                "traffic": (ratio * ab / nlaunch) if ratio is not None else None,
                "kernel": "double-float level kernels (per level or fused level pair the autotuned "
                          "k_level_stream ring, k_level_warp or k_level_fwd; every launch of the timed "
                          "region is one of them)",
                "algorithmic_bytes_per_launch": ab / nlaunch, "launches_per_apply": nlaunch}
    # end to end through the C call: pinned host x -> device, apply, device -> host y
    xh = torch.from_numpy(g.copy()).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    xdev = torch.empty_like(gd)
    ydev = torch.empty_like(gd)

    def e2e_step():
        xdev.copy_(xh, non_blocking=True)
        plan.apply(xdev, mode=P.MODE_DF64, out=ydev)
        yh.copy_(ydev, non_blocking=True)

    e2e_sec = timed_loop(e2e_step, args.steps, args.warmup, world, stream)
    e2e_value, _ = job_throughput(1.0, e2e_sec, world)
    if not torch.allclose(yh.cuda(), ydf):
        raise RuntimeError("end-to-end result differs from the device apply")
    line = {"metric": METRIC, "value": value, "unit": "applies/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32x2", "data": "synthetic",
            "config": {"workload": workload(N_LOG2), "N": N, "eps": EPS, "leaf": LEAF, "nrhs": 1,
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                       "l2": f"inputs larger than L2: {st['entries']*16/1e9:.1f} GB of factors per apply"},
            "rel_err": {"eps_a_fp64_vs_dense_256_rows": eps_a, "df64_vs_fp64": rel_df, "fp32_vs_fp64": rel_32},
            "roofline": roofline, "cpu_baseline": None,
            "e2e": {"value": e2e_value, "unit": "applies/s", "h2d_bytes_per_step": N * 16, "d2h_bytes_per_step": N * 16},
            "gpu_launches": nlaunch * args.steps, "clocks": clocks, "modes": modes, "autotune": tune,
            "library_peaks": lpk,
            "build": {"seconds": build_s, "entries": st["entries"], "levels": L + 1,
                      "level_kmax": st["level_kmax"], "level_entries": st["level_entries"],
                      "rank_saturated": st["rank_saturated"],
                      "device_GB": st["device_bytes"] / 1e9}}
    sub_steps = max(3, min(args.steps, 10))
    configs = {}
    if not args.headline_only and "fp32" in want:
        # differentiation on the same factorization (complex64 storage kept for the FP32 mode)
        configs["autograd"] = sub_autograd(plan, P, torch, inputs, sub_steps, args.warmup, world, lpk)
    plan.close()
    del plan, ybuf, y64, ydf, y32
    torch.cuda.empty_cache()
    if not args.headline_only:
        # the same construction with the IDs' QR in double-float (the headline plan used FP64)
        configs["build"] = sub_build(P, torch, inputs, N_LOG2, lpk, arith=("df64",))
        configs["build"]["fp64_qr_seconds_of_the_headline_plan"] = build_s
        configs["build"]["speedup_df64_vs_fp64_qr"] = build_s / configs["build"]["value"]
        torch.cuda.empty_cache()
        configs["mrhs"] = sub_mrhs(P, torch, inputs, 18, sub_steps, args.warmup, world, lpk)
        torch.cuda.empty_cache()
        configs["batch"] = sub_batch(P, torch, inputs, None, max(3, min(args.steps, 5)), args.warmup, world, lpk)
        torch.cuda.empty_cache()
        configs.update(sub_examples(P, torch, inputs, N_LOG2, sub_steps, args.warmup, world, lpk))
        torch.cuda.empty_cache()
    line["configs"] = configs
    if team is not None:
        times = team.run()
        line["cpu_baseline"] = cpu_summary(team, times, st["entries"])
    return line


def sub_autograd(plan, P, torch, inputs, steps, warmup, world, lpk, R=32):
    """Differentiation: loss ||K x - b||^2, complex FP32, R right-hand sides; the forward apply and
    the hand-written adjoint butterfly as torch.autograd backward."""
    N = plan.N
    X = torch.from_numpy(inputs.complex_gaussian(N, R, seed=5)).to(torch.complex64).cuda()
    B = torch.from_numpy(inputs.complex_gaussian(N, R, seed=6)).to(torch.complex64).cuda()
    out = {}

    def step():
        xv = X.clone().requires_grad_(True)
        loss = ((P.apply(plan, xv, P.MODE_FP32) - B).abs() ** 2).sum()
        loss.backward()
        out["loss"], out["g"] = loss, xv.grad

    sec = timed_loop(step, steps, warmup, world)
    value, tmax = job_throughput(1.0, sec, world)
    fma_pk = lpk["fp32_tflops"] / 2
    achieved = 8.0 * plan.stats()["entries"] * R / sec / 1e12  # forward + adjoint: 4 real FMA per entry and rhs each
    hbm_pk, hbm_kind = peaks()
    lbytes = 2 * plan.level_bytes(R, 8, 8)  # forward and adjoint, one launch per level each
    lg = N.bit_length() - 1
    return {"metric": f"IDBF forward+backward steps/s at N=2^{lg}, {R} RHS (loss ||Kx-b||^2, adjoint-butterfly backward)",
            "value": value, "unit": "fwd+bwd/s", "ms_per_step": tmax * 1e3, "steps": steps, "dtype": "f32",
            "workload": f"1D FIO N=2^{lg} eps=1e-6 leaf 64, {R} RHS complex64 (x seed 5, b seed 6)",
            "loss": float(out["loss"].detach()), "grad_norm": float(torch.linalg.norm(out["g"])),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fma_pk, "unit": "TFMA/s", "frac": achieved / fma_pk,
                         "peak_kind": "measured in this run: cuBLAS SGEMM 8192^3 (FP32, TF32 off) / 2 flops per FMA",
                         "hbm": {"achieved": lbytes / sec / 1e9, "peak": hbm_pk, "unit": "GB/s",
                                 "frac": lbytes / sec / 1e9 / hbm_pk, "peak_kind": hbm_kind,
                                 "bytes_per_step": lbytes}},
            "gradient_checks": "finite differences, dense K^* and gradcheck at N=4096 (tests/test_gpu_autograd.py)"}


def sub_mrhs(P, torch, inputs, log2n, steps, warmup, world, lpk, R=256):
    """Many right-hand sides: N = 2^18, eps = 1e-6, 256 RHS, complex FP32 factors. Timed: 3xTF32
    tensor cores on every level; the same with the middle factor S^h in double-float on the CUDA
    cores; the register-tiled FP32 CUDA-core apply (the same accuracy class without tensor cores);
    and the FP64 apply of the same 256 vectors. Errors against that FP64 apply."""
    N = 1 << log2n
    x, xi = inputs.uniform_grid(N)
    plan = P.Plan.build(x, xi, eps=EPS, leaf=LEAF, kernel="fio", c_profile=0, oversample=T_OVERSAMPLE,
                        oversample_leaf=T_LEAF)
    plan.set_storage(P.STORE_C128, P.STORE_C64)
    X = torch.from_numpy(inputs.complex_gaussian(N, R, seed=3)).cuda()
    X32 = X.to(torch.complex64)
    plan.reserve(R)
    y64 = plan.apply(X, mode=P.MODE_FP64)
    s64 = timed_loop(lambda: plan.apply(X, mode=P.MODE_FP64), 1, 1, world)
    hv = plan.L // 2
    for l in range(plan.L + 1):  # C64 everywhere; the middle level also in double-float
        plan.set_level_storage(l, *((P.STORE_DF64, P.STORE_C64) if l == hv else (P.STORE_C64,)))
    res = {}
    nrm = torch.linalg.norm(y64)
    for name, mode, n in (("tf32x3", P.MODE_TF32X3, steps), ("tf32x3_s64", P.MODE_TF32X3_S64, max(3, steps // 2)),
                          ("fp32_cuda_cores", P.MODE_FP32, steps)):
        yb = torch.empty_like(X32)
        sec = timed_loop(lambda: plan.apply(X32, mode=mode, out=yb), n, warmup, world)
        plan.sync_status()
        res[name] = {"ms_per_apply": sec * 1e3, "applies_per_s": 1.0 / sec,
                     "rel_err_vs_fp64": float(torch.linalg.norm(yb.to(torch.complex128) - y64) / nrm),
                     "speedup_vs_fp64": s64 / sec}
    st = plan.stats()
    lbytes = plan.level_bytes(R, 8, 8)     # complex64 factors and vectors
    hbm_pk, hbm_kind = peaks()
    useful = 8.0 * st["entries"] * R       # real flops of the complex block products
    executed = 3.0 * useful                # three split products on the tensor cores
    stc = res["tf32x3"]["ms_per_apply"] / 1e3
    value, tmax = job_throughput(1.0, stc, world)
    plan.close()
    return {"metric": f"IDBF multi-RHS applies/s at N=2^{log2n}, {R} RHS (3xTF32 tensor cores, error vs FP64 stated)",
            "value": value, "unit": f"applies/s ({R} rhs each)", "ms_per_step": tmax * 1e3, "steps": steps,
            "dtype": "tf32x3", "workload": f"1D FIO N=2^{log2n} eps=1e-6 leaf 64, {R} complex Gaussian RHS (seed 3), "
                                          "complex64 factors",
            "rel_err_vs_fp64": res["tf32x3"]["rel_err_vs_fp64"], "bar": "eps + 1e-6 = 2e-6",
            "vector_applies_per_s": value * R, "fp64_ms_per_apply": s64 * 1e3, "modes": res,
            # one launch per level: each reads its input boundary and writes its output boundary
            # (3.1 GB each at 256 right-hand sides), which outweighs the 5.5 GB of factors; the
            # tensor work (3 split products) would take 4.3 ms at the measured TF32 rate, the bytes
            # ~13 ms at the measured HBM rate: HBM is the bound of this unfused form
            "roofline": {"bound": "hbm", "achieved": lbytes / stc / 1e9, "unit": "GB/s", "peak": hbm_pk,
                         "frac": lbytes / stc / 1e9 / hbm_pk, "peak_kind": hbm_kind,
                         "bytes_per_apply": lbytes, "traffic": None,
                         "tensor": {"achieved": executed / stc / 1e12, "unit": "TFLOP/s", "peak": lpk["tf32_tflops"],
                                    "frac": executed / stc / 1e12 / lpk["tf32_tflops"],
                                    "peak_kind": "measured in this run: cuBLAS TF32 GEMM 8192^3",
                                    "useful_TFLOPs": useful / stc / 1e12}}}


def sub_batch(P, torch, inputs, cap_log2n, steps, warmup, world, lpk):
    """Uneven batch: 64 operators, N = 2^e with e uniform in [12, 18], the first half the FIO and
    the second half the jittered DFT kernel, 1-32 RHS each, eps = 1e-6. Timed in FP32 (the value)
    and double-float, each three ways: all 64 in one persistent launch in a CUDA graph (tiles
    autotuned); with the split autotuned too (operators from some N up run through their own
    per-level kernels after the launch; the value); and the same 64 applies made one plan at a
    time. Errors against the FP64 apply. FIO operators of equal N are the
    same matrix: the first is built, the others are device copies of it (idbf_clone), so that every
    operator still reads factor memory of its own."""
    ops = inputs.uneven_batch(seed=4)
    if cap_log2n is not None:  # a smaller batch for profiling: the same draw, N capped
        ops = [dict(o, N=min(o["N"], 1 << cap_log2n)) for o in ops]
    plans, xs, built = [], [], {}
    t0 = time.time()
    for o in ops:
        N = o["N"]
        if o["kind"] == "fio":
            if N in built:
                p = built[N].clone()
            else:
                x, xi = inputs.uniform_grid(N)
                p = P.Plan.build(x, xi, eps=EPS, leaf=LEAF, kernel="fio", c_profile=0, oversample=T_OVERSAMPLE,
                                 oversample_leaf=T_LEAF)
                built[N] = p
        else:
            x, xi = inputs.jittered_grid(N, seed=o["seed"])
            p = P.Plan.build(x, xi, eps=EPS, leaf=LEAF, kernel="dft", sign=-1)
        plans.append(p)
        xs.append(torch.from_numpy(inputs.complex_gaussian(N, o["nrhs"], seed=o["seed"])).cuda())
    build_s = time.time() - t0
    y64 = [p.apply(x, mode=P.MODE_FP64) for p, x in zip(plans, xs)]
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
        # every operator in the one persistent launch (tiles autotuned)
        # a double-float batch takes 1-2 s and repeats to 0.1 %: fewer trials and steps there
        reps = 1 if name == "df64" else 2
        st_, wu_ = (min(steps, 3), min(warmup, 3)) if name == "df64" else (steps, warmup)
        b.set_split(P.Batch.NO_SPLIT)
        one_tuned = b.autotune(xm, reps=reps)
        one = timed_loop(lambda: b.apply(xm, ym), st_, wu_, world)
        one_tiles = b.info()
        b.sync_status()
        # the autotuner also chooses the size above which operators run through their own applies
        b.set_split(0)
        tuned_ms = b.autotune(xm, reps=reps)
        secs = timed_loop(lambda: b.apply(xm, ym), st_, wu_, world)
        b.sync_status()
        err = max(float(torch.linalg.norm(y.to(torch.complex128) - r) / torch.linalg.norm(r)) for y, r in zip(ym, y64))
        sep = timed_loop(lambda: [p.apply(x, mode=mode) for p, x in zip(plans, xm)], max(1, steps // 2), 1, world)
        algo = sum(p.algorithmic_bytes(x.shape[1], eb, eb) for p, x in zip(plans, xs))
        fma = sum(4.0 * p.stats()["entries"] * x.shape[1] for p, x in zip(plans, xs))  # real FMA per complex MAC: 4
        res[name] = {"ms_per_batch": secs * 1e3, "batches_per_s": 1.0 / secs, "algorithmic_GBps": algo / secs / 1e9,
                     "useful_TFMA_per_s": fma / secs / 1e12,
                     "algorithmic_bytes": algo, "max_rel_err_vs_fp64": err, "tiles": b.info(), "split": b.split(),
                     "autotune_best_ms": tuned_ms, "separate_applies_ms": sep * 1e3,
                     "speedup_vs_separate_applies": sep / secs,
                     "one_launch": {"ms_per_batch": one * 1e3, "tiles": one_tiles, "autotune_best_ms": one_tuned,
                                    "speedup_vs_separate_applies": sep / one}}
        b.close()
    for p in plans:
        p.close()
    value, tmax = job_throughput(1.0, res["fp32"]["ms_per_batch"] / 1e3, world)
    peak, kind = peaks()
    fma_pk = lpk["fp32_tflops"] / 2
    r32 = res["fp32"]
    return {"metric": "IDBF uneven-batch applies/s (64 operators, N 2^12..2^18, 1-32 RHS; one persistent launch in a "
                      "CUDA graph for the operators below an autotuned size split, their own per-level launches above)",
            "value": value, "unit": "batches/s (64 operator applies each)", "ms_per_step": tmax * 1e3, "steps": steps,
            "dtype": "f32",
            "workload": "64 ops, seed 4: FIO (ops 0-31) / jittered DFT (32-63), eps=1e-6, leaf 64, complex64 factors"
                        + (f", N capped at 2^{cap_log2n}" if cap_log2n is not None else ""),
            "rel_err": {"max_over_ops_vs_fp64": r32["max_rel_err_vs_fp64"]},
            "operator_applies_per_s": 64 * value, "vector_applies_per_s": sum(o["nrhs"] for o in ops) * value,
            # 1-32 right-hand sides make ~8 FMA per factor byte: the FP32 FMA pipes, not HBM, bound it
            "roofline": {"bound": "alu", "achieved": r32["useful_TFMA_per_s"], "peak": fma_pk, "unit": "TFMA/s",
                         "frac": r32["useful_TFMA_per_s"] / fma_pk,
                         "peak_kind": "measured in this run: cuBLAS SGEMM 8192^3 / 2 flops per FMA",
                         "hbm_GBps": r32["algorithmic_GBps"], "hbm_frac_of_measured": r32["algorithmic_GBps"] / peak},
            "modes": res, "build_seconds_total": build_s, "distinct_builds": len(built) + 32,
            "N": [o["N"] for o in ops], "nrhs": [o["nrhs"] for o in ops]}


def sub_build(P, torch, inputs, log2n, lpk, arith=("fp64", "df64")):
    """The on-device construction (idbf_build) of the benchmarked FIO at N = 2^log2n with the IDs'
    pivoted QR in FP64 and in double-float arithmetic: seconds, stored entries and eps^a of Sec. 3
    on 256 rows against GPU direct rows (not part of the apply metric). The line's value is the
    time of the last arithmetic listed."""
    N = 1 << log2n
    x, xi = inputs.uniform_grid(N)
    g = torch.from_numpy(inputs.complex_gaussian(N, 1, seed=SEED)[:, 0]).cuda()
    rows = torch.from_numpy(inputs.sample_rows(N, 256, seed=SEED)).cuda()
    ud = P.kernel_matvec_rows(torch.from_numpy(x).cuda(), torch.from_numpy(xi).cuda(), g, rows, kernel="fio",
                              c_profile=0)
    res = {}
    for name in arith:
        torch.cuda.synchronize()
        t0 = time.time()
        plan = P.Plan.build(x, xi, eps=EPS, leaf=LEAF, kernel="fio", c_profile=0, oversample=T_OVERSAMPLE,
                            oversample_leaf=T_LEAF, qr_arith=P.QR_DF64 if name == "df64" else P.QR_FP64)
        torch.cuda.synchronize()
        secs = time.time() - t0
        st = plan.stats()
        y = plan.apply(g)
        eps_a = float(torch.linalg.norm(y[rows] - ud) / torch.linalg.norm(ud))
        res[name] = {"seconds": secs, "entries": st["entries"], "level_kmax": st["level_kmax"],
                     "rank_saturated": st["rank_saturated"], "eps_a_256_rows": eps_a}
        plan.close()
        del y
        torch.cuda.empty_cache()
    last = res[arith[-1]]
    out = {"metric": f"IDBF on-device build seconds at N=2^{log2n} (FIO, eps=1e-6, leaf 64, {arith[-1]} QR)",
           "value": last["seconds"], "unit": "s", "ms_per_step": last["seconds"] * 1e3, "steps": 1, "dtype": "f64",
           "higher_is_better": False,
           "workload": f"1D FIO N=2^{log2n} eps=1e-6 leaf 64, Mock-Chebyshev t=2 (t=4 at the leaf)",
           "qr": res, "fp64_peak_TFLOPs": lpk["fp64_tflops"]}
    if "fp64" in res and "df64" in res:
        out["speedup_df64_vs_fp64_qr"] = res["fp64"]["seconds"] / res["df64"]["seconds"]
    return out


def sub_examples(P, torch, inputs, log2n, steps, warmup, world, lpk):
    """The paper's other two workloads at N = 2^log2n, built on the GPU (double-float QR) and
    applied to one vector: Example 2, the Schloemilch expansion J_0(x xi) on x_k = (k-1)/N,
    xi_n = n pi; Example 3, the non-uniform DFT exp(-2 pi i omega x) on N random omega in
    [-N/2, N/2) and N random x in [0, 1), on coordinate-based dyadic trees (leaves of uneven size,
    about 64 points each). Per example: build seconds, stored entries, eps^a of Sec. 3 on 256 rows
    against GPU direct rows (FP64 apply), and the double-float and FP32 applies (autotuned per
    level) with their errors against the FP64 apply and their HBM figures: algorithmic bytes
    (factors, indices, x and y once) and level bytes (plus each boundary written and read back)
    per second, against the measured copy bandwidth."""
    import numpy as np
    N = 1 << log2n
    hbm_pk, hbm_kind = peaks()
    out = {}
    g = torch.from_numpy(inputs.complex_gaussian(N, 1, seed=SEED)[:, 0]).cuda()
    g32 = g.to(torch.complex64)
    rows = torch.from_numpy(inputs.sample_rows(N, 256, seed=SEED)).cuda()
    for name in ("ex2_schlomilch_j0", "ex3_nufft_random_points"):
        torch.cuda.synchronize()
        t0 = time.time()
        if name.startswith("ex2"):
            x, xi = inputs.schlomilch_grid(N)
            kern, sign = "j0", -1
            # J_0 needs more sampled rows than the FIO for the same accuracy (t = 2 gives eps^a
            # ~18 eps at N = 2^20, t = 4 ~5 eps, at the same ranks)
            plan = P.Plan.build(x, xi, eps=EPS, leaf=LEAF, kernel=kern, oversample=2 * T_OVERSAMPLE,
                                oversample_leaf=2 * T_LEAF, qr_arith=P.QR_DF64)
            desc = (f"Example 2: J_0(x xi), x_k=(k-1)/N, xi_n=n pi, N=2^{log2n}, eps=1e-6, leaf 64, "
                    f"Mock-Chebyshev t=4 (t=8 at the leaf)")
        else:
            x, xi = inputs.nufft_points(N, seed=N)   # x: the row points omega, xi: the column points
            kern, sign = "dft", -1
            L = P.tree_depth(N, LEAF)
            ro, co = P.dyadic_leaves(x, -N / 2, N / 2, L), P.dyadic_leaves(xi, 0.0, 1.0, L)
            plan = P.Plan.build_leaves(x, xi, L, ro, co, eps=EPS, kernel=kern, sign=sign, oversample=T_OVERSAMPLE,
                                       oversample_leaf=T_LEAF, qr_arith=P.QR_DF64)
            desc = (f"Example 3: exp(-2 pi i omega x), N=2^{log2n} random omega in [-N/2,N/2) and x in [0,1) "
                    f"(seed N), dyadic trees of depth {L}, leaves of uneven size (mean 64), eps=1e-6, "
                    f"Mock-Chebyshev t=2 (t=4 at the leaf)")
        torch.cuda.synchronize()
        build_s = time.time() - t0
        plan.set_storage(P.STORE_C128, P.STORE_DF64, P.STORE_C64)
        st = plan.stats()
        y64 = plan.apply(g, mode=P.MODE_FP64)
        ud = P.kernel_matvec_rows(torch.from_numpy(np.ascontiguousarray(x)).cuda(),
                                  torch.from_numpy(np.ascontiguousarray(xi)).cuda(), g, rows, kernel=kern, sign=sign)
        eps_a = float(torch.linalg.norm(y64[rows] - ud) / torch.linalg.norm(ud))
        nrm = torch.linalg.norm(y64)
        modes = {}
        for mname, mode, vec, eb in (("df64", P.MODE_DF64, g, 16), ("fp32", P.MODE_FP32, g32, 8)):
            plan.autotune(mode, reps=10)
            yb = torch.empty_like(vec)
            sec = timed_loop(lambda: plan.apply(vec, mode=mode, out=yb), steps, warmup, world)
            ab, lb = plan.algorithmic_bytes(1, eb, eb), plan.level_bytes(1, eb, eb)
            modes[mname] = {"applies_per_s": 1.0 / sec, "ms_per_apply": sec * 1e3,
                            "rel_err_vs_fp64": float(torch.linalg.norm(yb.to(torch.complex128) - y64) / nrm),
                            "algorithmic_GBps": ab / sec / 1e9, "level_GBps": lb / sec / 1e9,
                            "frac_of_hbm_algorithmic": ab / sec / 1e9 / hbm_pk,
                            "level_variants": plan.stats()["level_variant"][P.STORE_DF64 if mname == "df64" else P.STORE_C64]}
        s64 = timed_loop(lambda: plan.apply(g, mode=P.MODE_FP64), max(3, steps // 2), warmup, world)
        modes["fp64"] = {"applies_per_s": 1.0 / s64, "ms_per_apply": s64 * 1e3}
        value, tmax = job_throughput(1.0, modes["df64"]["ms_per_apply"] / 1e3, world)
        out[name] = {"metric": f"IDBF applies/s, {name}, double-float, 1 RHS", "value": value, "unit": "applies/s",
                     "ms_per_step": tmax * 1e3, "steps": steps, "dtype": "f32x2", "workload": desc,
                     "build": {"seconds": build_s, "qr": "df64", "entries": st["entries"], "levels": st["L"] + 1,
                               "level_kmax": st["level_kmax"], "device_GB": st["device_bytes"] / 1e9},
                     "eps_a_fp64_vs_direct_256_rows": eps_a, "modes": modes,
                     "roofline": {"bound": "hbm", "achieved": modes["df64"]["algorithmic_GBps"], "unit": "GB/s",
                                  "peak": hbm_pk, "frac": modes["df64"]["frac_of_hbm_algorithmic"],
                                  "peak_kind": hbm_kind, "traffic": None}}
        plan.close()
        del y64
        torch.cuda.empty_cache()
    return out


def single_line(sub, args, world):
    """One JSON line for a workload run on its own (--workload mrhs | batch | autograd)."""
    line = {"metric": sub["metric"], "value": sub["value"], "unit": sub["unit"], "n_gpus": world,
            "steps": sub["steps"], "warmup": args.warmup, "ms_per_step": sub["ms_per_step"],
            "higher_is_better": sub.get("higher_is_better", True), "scaling": "weak", "vs_baseline": None,
            "dtype": sub["dtype"],
            "data": "synthetic", "config": {"workload": sub["workload"]}}
    line.update({k: v for k, v in sub.items() if k not in line and k != "workload"})
    return line


def gpu_workload(args, rank, world):
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_1809_10573_gb300 as P
    from paper_1809_10573_gb300 import inputs
    lpk = library_peaks()
    steps = args.steps
    if args.workload == "mrhs":
        sub = sub_mrhs(P, torch, inputs, args.log2n if args.log2n is not None else 18, steps, args.warmup, world, lpk)
    elif args.workload == "batch":
        sub = sub_batch(P, torch, inputs, args.log2n, steps, args.warmup, world, lpk)
    elif args.workload == "build":
        sub = sub_build(P, torch, inputs, args.log2n if args.log2n is not None else 20, lpk)
    elif args.workload == "examples":
        subs = sub_examples(P, torch, inputs, args.log2n if args.log2n is not None else 20, steps, args.warmup, world,
                            lpk)
        if rank == 0:
            for sub in subs.values():
                line = single_line(sub, args, world)
                line["library_peaks"] = lpk
                print(json.dumps(line), flush=True)
        return 0
    else:
        N = 1 << (args.log2n if args.log2n is not None else 20)
        x, xi = inputs.uniform_grid(N)
        plan = P.Plan.build(x, xi, eps=EPS, leaf=LEAF, kernel="fio", c_profile=0, oversample=T_OVERSAMPLE,
                            oversample_leaf=T_LEAF)
        plan.set_storage(P.STORE_C64)
        sub = sub_autograd(plan, P, torch, inputs, steps, args.warmup, world, lpk)
    if rank == 0:
        line = single_line(sub, args, world)
        line["library_peaks"] = lpk
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
    ap.add_argument("--workload", choices=["apply", "mrhs", "batch", "autograd", "build", "examples"], default="apply",
                    help="apply (default): the headline single-vector apply at N=2^20, with the multi-RHS, batch "
                         "and autograd workloads as sub-objects of its line; the others print a line of their own")
    ap.add_argument("--headline-only", action="store_true",
                    help="apply workload without the multi-RHS, batch and autograd sub-objects (profiling)")
    args = ap.parse_args()
    global N_LOG2
    N_LOG2 = args.log2n if args.log2n is not None else 20
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")
    rank, world, local = dist_init()
    try:
        if args.impl == "reference":
            return cpu_arm(args, rank, world)
        if args.workload != "apply":
            return gpu_workload(args, rank, world)
        return gpu_arm(args, rank, world, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
