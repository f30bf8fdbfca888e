"""Host logic of bench.py's multi-process mode on CPU (gloo, world size 2): the whole-job
time is the maximum over ranks, and the reference arm prints from rank 0 only."""
import json
import os
import socket
import subprocess
import sys

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


def test_traffic_record_voided_by_source_change(tmp_path, monkeypatch):
    """The roofline's DRAM-traffic figure comes from a committed ncu record only while the
    squaring kernel's sources hash to the value stored with it; any change voids it (null)."""
    import shutil
    sys.path.insert(0, ROOT)
    import bench
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic_sp2_square_tc_fp16x6_lattice32.json")))
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    shutil.copy(os.path.join(ROOT, "profiles", "traffic_sp2_square_tc_fp16x6_lattice32.json"), root / "profiles")
    for src in rec["sources"]:
        (root / src).parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(ROOT, src), root / src)
    monkeypatch.setattr(bench, "ROOT", str(root))
    t = bench.captured_traffic("sp2_square_tc_fp16x6", "lattice32")
    assert t == sum(rec["dram_bytes_per_launch"]) / len(rec["dram_bytes_per_launch"])
    with open(root / rec["sources"][0], "a") as f:
        f.write("\n// changed\n")
    assert bench.captured_traffic("sp2_square_tc_fp16x6", "lattice32") is None
    assert bench.captured_traffic("sp2_square_tc_fp16x6", "no_such_workload") is None
