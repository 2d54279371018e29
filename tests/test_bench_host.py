"""Host-side logic of bench.py: whole-job throughput over ranks (gloo, world size 2 on CPU),
the clock-record parsing, and the traffic summary's validity check."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    secs = [2.0, 3.0][rank]                  # the slower rank decides
    value, t = bench.job_throughput(10, secs, world)
    bench.barrier(world)
    q.put((rank, value, t))
    dist.destroy_process_group()


def test_job_throughput_takes_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for _, value, t in out:
        assert t == 3.0 and abs(value - 20 / 3.0) < 1e-12


def test_single_rank_throughput():
    assert bench.job_throughput(5, 2.0, 1) == (2.5, 2.0)


def test_clock_summary_parsing(tmp_path):
    cs = bench.ClockSampler(0)
    f = tmp_path / "c.csv"
    f.write_text("2026/12/03 01:00:00.000, 0, 1900, 2070, 900.5, 0x4, Not Active, Not Active, Not Active, Active\n"
                 "2026/12/03 01:00:00.200, 0, 1950, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    cs.f = open(f, "r+")
    s = cs.summary()
    assert s["samples"] == 2 and s["sm_mhz"] == 1925 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["sw_power_cap"]


def test_traffic_summary_requires_the_profiled_source(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "paper_1809_10573_gb300" / "csrc").mkdir(parents=True)
    src = "int f(int a) {  // one\n  /* two */ return a + 1;\n}\n"
    (tmp_path / "paper_1809_10573_gb300" / "csrc" / "apply.cu").write_text(src)
    (tmp_path / "profiles" / "level_kernel_traffic.txt").write_text(
        "# c\ndram_bytes_per_algorithmic_byte = 1.25\napply_cu_code_sha256 = " + bench.code_digest(src) + "\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.read_traffic_summary() == 1.25
    # a comment edit keeps the figure, a code edit voids it
    (tmp_path / "paper_1809_10573_gb300" / "csrc" / "apply.cu").write_text(
        "int f(int a) {  // changed comment\n\n  /* x\n y */ return a + 1;\n}\n")
    assert bench.read_traffic_summary() == 1.25
    (tmp_path / "paper_1809_10573_gb300" / "csrc" / "apply.cu").write_text("int f(int a) { return a + 2; }\n")
    assert bench.read_traffic_summary() is None


def test_level_variants_option_parsing():
    assert bench.parse_level_variants(None) == {}
    assert bench.parse_level_variants("df64=14,1,10") == {"df64": [14, 1, 10]}
    assert bench.parse_level_variants(" df64=7,1 ; fp32=3,15 ;") == {"df64": [7, 1], "fp32": [3, 15]}
    with pytest.raises(ValueError):
        bench.parse_level_variants("df64=7,x")


def test_launches_per_apply_counts_fused_pairs_once():
    # a pair variant (16-19) on level l < L covers levels l and l + 1; on level L it is one level
    assert bench.launches_per_apply([1] * 15, 14) == 15
    assert bench.launches_per_apply([19, 19, 14, 1, 1, 1, 1, 5, 1, 10, 14], 10) == 10
    assert bench.launches_per_apply([16, 3, 17, 0, 1], 4) == 3
    assert bench.launches_per_apply([0, 1, 16], 2) == 3
    assert bench.launches_per_apply([0, 16, 16], 2) == 2


def test_oracle_team_times_one_core_then_all(monkeypatch):
    """The CPU baseline's worker processes (spawned: no CUDA state is inherited) build the oracle's
    factorization, then run the single-core and the all-core phases in lockstep with the parent."""
    team = bench.OracleTeam(2, 9, steps_single=2, steps_all=3)
    try:
        times = team.run()
    finally:
        team.close()
    assert [len(t) for t in times] == [2, 3] and all(v > 0 for t in times for v in t)
    assert team.entries > 0
    cb = bench.cpu_summary(team, times, 100 * team.entries)
    assert cb["cores"] == 2 and cb["kind"] == "oracle" and cb["single_core"]["cores"] == 1
    # two processes each applying once per step, entries scaled by 100
    assert abs(cb["value"] - 2 / (sorted(times[1])[1] * 100)) < 1e-9 * cb["value"]


def test_reference_arm_prints_one_measured_line(monkeypatch, capsys):
    import argparse
    import json
    monkeypatch.setattr(bench, "CPU_LOG2", 9)
    monkeypatch.setattr(bench, "host_cores", lambda: 2)
    args = argparse.Namespace(gpus=1, steps=3, warmup=3)
    assert bench.cpu_arm(args, 0, 1) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["cpu_baseline"]["cores"] == 2
    # ms_per_step is the wall time a step really took: the timed steps fit the run
    assert line["ms_per_step"] * line["steps"] < 60e3
    assert line["e2e"]["value"] == line["value"]
