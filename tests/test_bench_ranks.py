"""Host logic of bench.py on CPU: in multi-process mode (gloo, world size 2) the whole-job
time is the maximum over ranks, the reference arm prints from rank 0 only, and a clock
record that voids a timing on any rank makes every rank measure again; the nvidia-smi
clock summary and its verdict; the traffic record's tie to the kernel sources."""
import json
import os
import socket
import subprocess
import sys
import time

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = bench.max_over_ranks(1.5 + 2.0 * rank, world)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        assert dict(out) == {0: 3.5, 1: 3.5}


def test_reference_arm_prints_on_rank0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_line():
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "orbitals/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    # the base contract's keys, with the GPU arm's metric, unit and direction
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config"):
        assert key in d, key
    sys.path.insert(0, ROOT)
    import bench
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["n_gpus"] == 1 and d["config"]["workload"].startswith("lattice32")
    assert d["e2e"]["value"] == d["value"] == d["cpu_baseline"]["value"]


def test_traffic_record_voided_by_source_change(tmp_path, monkeypatch):
    """The roofline's DRAM-traffic figure comes from a committed ncu record only while the
    squaring kernel's sources hash to the value stored with it; any change voids it (null).
    The record here is a stand-in written for the current sources in a scratch copy."""
    import hashlib
    import shutil
    sys.path.insert(0, ROOT)
    import bench
    srcs = bench.TRAFFIC_SOURCES["sp2_square_tc_fp16x6"]
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    h = hashlib.sha256()
    for src in srcs:
        (root / src).parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(ROOT, src), root / src)
        h.update(open(os.path.join(ROOT, src), "rb").read())
    rec = {"kernel": "sp2_square_tc_fp16x6", "workload": "lattice32", "dram_bytes_per_launch": [100, 300],
           "sources": srcs, "sha256": h.hexdigest(), "capture": "stand-in"}
    with open(root / "profiles" / "traffic_sp2_square_tc_fp16x6_lattice32.json", "w") as f:
        json.dump(rec, f)
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.captured_traffic("sp2_square_tc_fp16x6", "lattice32") == 200
    with open(root / srcs[0], "a") as f:
        f.write("\n// changed\n")
    assert bench.captured_traffic("sp2_square_tc_fp16x6", "lattice32") is None
    assert bench.captured_traffic("sp2_square_tc_fp16x6", "no_such_workload") is None


def _smi(sm, smax, hw="Not Active", hwt="Not Active", swt="Not Active", pcap="Not Active"):
    """One line of nvidia-smi's CSV for the sampler's query (noheader, nounits)."""
    return "0, %s, %s, 1100.5, 0x0, %s, %s, %s, %s" % (sm, smax, hw, hwt, swt, pcap)


def test_clock_summary_and_verdict():
    sys.path.insert(0, ROOT)
    import bench
    lines = [_smi(2070, 2070), _smi(1980, 2070, pcap="Active"), _smi(2055, 2070), "garbage", "",
             _smi("[N/A]", 2070), "0, 2070, 2070"]
    clk = bench.summarize_clock_lines(lines)
    assert clk == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert bench.clock_verdict(clk) is None                      # the power cap is kept, not rejected
    for field in ("hw", "hwt", "swt"):
        c = bench.summarize_clock_lines([_smi(2070, 2070), _smi(1900, 2070, **{field: "Active"})])
        assert bench.clock_verdict(c).startswith("throttled: ")
    stuck = bench.summarize_clock_lines([_smi(1200, 2070)] * 5)
    assert stuck["reasons"] == [] and "1200 of 2070" in bench.clock_verdict(stuck)
    # a low clock with a reason reported is the power cap's doing, not a lock
    assert bench.clock_verdict(bench.summarize_clock_lines([_smi(1500, 2070, pcap="Active")] * 5)) is None
    assert bench.summarize_clock_lines([]) == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
    assert bench.clock_verdict({"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}) is None


def _verdict_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # only rank 1 saw a slowdown: both ranks must take the re-measure branch together
        clk = bench.summarize_clock_lines([_smi(2070, 2070, hwt="Active" if rank == 1 else "Not Active")])
        why = bench.clock_verdict(clk)
        out[rank] = bench.max_over_ranks(1.0 if why else 0.0, world) > 0
    finally:
        dist.destroy_process_group()


def test_remeasure_decision_is_collective():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_verdict_worker, args=(2, free_port(), out), nprocs=2, start_method="spawn")
        assert dict(out) == {0: True, 1: True}


def test_clock_sampler_with_fake_smi(tmp_path, monkeypatch):
    """The sampler against a stand-in nvidia-smi on PATH: it waits for the first sample,
    drops what was read before the region, and summarises what came during it."""
    sys.path.insert(0, ROOT)
    import bench
    fake = tmp_path / "nvidia-smi"
    # the first line (read before the region opens) reports a slowdown that must not count
    fake.write_text("#!/bin/sh\n"
                    "echo '%s'\n"
                    "while true; do echo '%s'; sleep 0.05; done\n"
                    % (_smi(900, 2070, hwt="Active"), _smi(2070, 2070, pcap="Active")))
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ["PATH"])
    s = bench.ClockSampler(0)
    s.start()
    assert s.first.is_set()
    time.sleep(0.5)
    clk = s.stop()
    assert clk["samples"] >= 3 and clk["sm_mhz"] == 2070.0 and clk["reasons"] == ["sw_power_cap"]
    assert bench.clock_verdict(clk) is None
    assert s.proc.poll() is not None
    # no nvidia-smi at all: the record says so and voids nothing
    monkeypatch.setenv("PATH", str(tmp_path / "empty"))
    s = bench.ClockSampler(0)
    s.start()
    clk = s.stop()
    assert clk["reasons"] == ["nvidia-smi unavailable"] and bench.clock_verdict(clk) is None


def test_ell_rows_diff_against_dense():
    """bench.ell_rows_diff (the D comparison of the mlp workloads' graphs) against the dense
    difference: ELL rows with different patterns and widths, entries absent on one side
    counting as zero, only the selected rows compared."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    rng = np.random.default_rng(3)
    n = 40

    def random_ell(width, fill):
        col = np.full((n, width), -1, dtype=np.int32)
        val = np.zeros((n, width))
        for i in range(n):
            k = rng.integers(1, min(fill, width) + 1)
            col[i, :k] = rng.choice(n, k, replace=False)
            val[i, :k] = rng.normal(size=k)
        return col, val

    def dense(col, val):
        D = np.zeros((n, n))
        for i in range(n):
            m = col[i] >= 0
            D[col[i][m], i] = val[i][m]
        return D

    ca, va = random_ell(12, 12)
    cb, vb = random_ell(20, 18)
    rows = np.sort(rng.choice(n, 25, replace=False))
    dd = (dense(ca, va) - dense(cb, vb))[:, rows]
    both = ((dense(ca, np.where(ca >= 0, 1.0, 0.0)) + dense(cb, np.where(cb >= 0, 1.0, 0.0))) > 0)[:, rows]
    t = torch.from_numpy
    mx, ss, cnt = bench.ell_rows_diff(torch, t(rows), t(ca), t(va), t(cb), t(vb), n, chunk=7)
    assert mx == np.abs(dd).max() and cnt == int(both.sum())
    assert abs(ss - float((dd ** 2).sum())) < 1e-12 * max(1.0, ss)
    assert bench.ell_rows_diff(torch, t(rows), t(ca), t(va), t(ca), t(va), n)[:2] == (0.0, 0.0)
    assert bench.mlp_init_params(0).shape == (4609,)
