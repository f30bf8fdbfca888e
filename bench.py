#!/usr/bin/env python
"""Benchmark: graph-partitioned SP2 density-matrix throughput on GB300.

Metric (one JSON line on rank 0): SP2 density-matrix orbitals/s = N / (gather + SP2 +
assembly time) of one D build, for the tensor-core FP16X6 path, with the FP64 GPU path,
tensor TFLOP/s, max |dD| between the two, a live roofline figure of the dominant kernel,
an end-to-end figure through the C ABI with host buffers, and the CPU oracle timed on a
bounded sample of the same workload.

Default workload: 32^3 jittered rock-salt lattice (N = 32768, seed 0), H_ij =
-exp(-(r-a)/0.3a) for r < 2.5a, graph |H^2| >= 0.15 (the knob that gives the stated
300-600 submatrix range), 512 cores of 4x4x4 sites from 8x8x8 spatial cells,
one global SP2 with FP64 global traces deciding every branch on the device, stop on
stalled idempotency error (n_min 10) or 1e-10.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gbe|reference]
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "SP2 density-matrix orbitals/s and tensor TFLOP/s, mixed vs FP64 at max|ΔD|≤1e-6"
UNIT = "orbitals/s"
WORKLOADS = {
    # the configuration the metric is quoted on: 32^3 lattice, cores of 64, m_s ~ 460-480
    "lattice32": dict(kind="lattice", L=32, seed=0, thresh=0.15, ncell=(8, 8, 8)),
    # the same lattice with the partition size chosen by gbe_partition_autotune among cell
    # grids of 4^3 .. 32^3 (cores of 512 .. 1 sites) by the modelled squaring time per SP2 step
    "lattice32tuned": dict(kind="lattice", L=32, seed=0, thresh=0.15, ncell=(8, 8, 8),
                           ncell_candidates=[(4, 4, 4), (8, 8, 8), (16, 16, 16), (32, 32, 32)]),
    # small case (8^3, |H^2| >= 1e-5 graph, cores of 8, m_s ~ 470-510)
    "lattice8": dict(kind="lattice", L=8, seed=0, thresh=1e-5, ncell=(4, 4, 4)),
    # 16^3 slice of the 32^3 workload (same m_s distribution, 64 subgraphs): profiling case
    "lattice16": dict(kind="lattice", L=16, seed=0, thresh=0.15, ncell=(4, 4, 4)),
    # disordered liquid-like system: 131072 uniform random sites (box 50.8a), cores of ~60
    # sites from 13^3 cells, |H^2| >= 0.1 halos: uneven m_s over several 128-wide buckets
    "disordered131k": dict(kind="disordered", N=131072, seed=0, thresh=0.1, ncell=(13, 13, 13), n_max=80),
    # 4096-site sample of the same model (box 16a, 4^3 cells): profiling / oracle sample
    "disordered4k": dict(kind="disordered", N=4096, seed=0, thresh=0.1, ncell=(4, 4, 4), n_max=80),
    # QMD-like run on the 32^3 lattice: positions advance by N(0, 0.01a) per step, the graph
    # comes from the previous step's |D| >= 1e-2 (first step: |H^2| >= 0.15), the SP2
    # sequence is the previous step's, replayed (no trace exchange during a step)
    "qmd32": dict(kind="lattice", L=32, seed=0, thresh=0.15, ncell=(8, 8, 8), qmd=True, tau=1e-2),
    # QMD-like run of the 16^3 lattice on its complete graph (one subgraph of all 4096 sites,
    # where SP2 converges and the gap estimate has its window): each step's branch sequence
    # comes from the HOMO-LUMO gap estimated at the previous step (Sec. II.C), FP64-grade;
    # the estimate reads the traces where the idempotency error is 1e-6 .. 1e-2, above the
    # FP64TC squarings' floor (~1e-9 over 4096 core positions)
    "qmd16gap": dict(kind="lattice", L=16, seed=0, qmd=True, complete=True, sequence="gap", prec="fp64tc",
                     gap_window=(1e-6, 1e-2), seq_tol=1e-12),
    # finite temperature on the 32^3 workload: Fermi function at kT = 0.25 eV (beta = 4/eV),
    # mu = 0, Chebyshev order 300 (coefficients below 1e-8 beyond it for this spectral width)
    "foe32": dict(kind="lattice", L=32, seed=0, thresh=0.15, ncell=(8, 8, 8), foe=dict(beta=4.0, mu=0.0, order=300)),
    # learned graph proposal at 1,048,576 disordered sites (box 101.6a): candidate pairs
    # r < 4a with features, the width-64 network over every pair, selection + union with H
    # learned graph proposal at 1,048,576 disordered sites (box 101.6a): the network is trained
    # on seeded 4096-site systems of the same model (box 16a; labels |D_ij| >= 1e-2 from the
    # library's FP64-grade SP2 on each one's complete graph), then proposes the graph of the
    # big system, whose FP64-grade graph SP2 is compared with the H^1 and H^2 pattern graphs'
    # (cores from 25^3 cells of ~67 sites, the branch sequence of one global-trace run replayed
    # on every graph, subgraphs in batches that fit the device)
    "mlp1m": dict(kind="disordered", N=1 << 20, seed=2024,
                  mlp=dict(rcand=4.0, cut=-2.0, cuts=(-6.0, -4.0, -2.0), tau=1e-2, train_n=4096, train_seed0=1000,
                           test_seed=1999, passes=40, lr=3e-3, ncell=(25, 25, 25), n_max=100)),
    # the same at 65,536 sites (box 40.3a, cores from 10^3 cells): a quick case of the pipeline
    "mlp64k": dict(kind="disordered", N=1 << 16, seed=2024,
                   mlp=dict(rcand=4.0, cut=-2.0, cuts=(-6.0, -4.0, -2.0), tau=1e-2, train_n=4096, train_seed0=1000,
                            test_seed=1999, passes=40, lr=3e-3, ncell=(10, 10, 10), n_max=100)),
}
PRECS = {"fp16x6": ("FP16X6", "f16-split(x6)/f32-acc/f64-trace"),
         "bf16x3": ("BF16X3", "bf16-split(x3)/f32-acc/f64-trace"),
         "fp64tc": ("FP64TC", "f16-fixed-point-slices(x18 products)/f32-acc, FP64-grade")}


def make_system(wl, seed):
    import synth
    if wl["kind"] == "lattice":
        return synth.lattice(wl["L"], seed=seed)
    return synth.disordered(wl["N"], seed=seed)
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def captured_traffic(kernel, workload):
    """DRAM bytes per launch from the committed ncu capture of this kernel and workload, or
    None when the kernel's sources changed since the capture (hash recorded with it)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic_%s_%s.json" % (kernel, workload))
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    h = hashlib.sha256()
    for src in d["sources"]:
        with open(os.path.join(ROOT, src), "rb") as f:
            h.update(f.read())
    if h.hexdigest() != d["sha256"]:
        return None
    return sum(d["dram_bytes_per_launch"]) / len(d["dram_bytes_per_launch"])


TRAFFIC_SOURCES = {
    "sp2_square_tc_fp16x6": ["paper_1603_00937_gb300/csrc/sp2_tc.cu", "paper_1603_00937_gb300/csrc/split.cuh",
                             "paper_1603_00937_gb300/csrc/gbe_internal.h"],
}
TRAFFIC_KERNEL_RE = {"sp2_square_tc_fp16x6": r"sp2_square_tc_kernel<1, (0|false)(, \d+)*>"}   # <FP16X6, FOE = false, ring depth, K-chunk>


def record_traffic(report, kernel, workload, capture_md):
    """Write profiles/traffic_<kernel>_<workload>.json from an ncu report of that workload:
    dram__bytes_read.sum + dram__bytes_write.sum of every captured launch of the kernel, with
    the hash of its sources (a later change of them voids the record)."""
    import csv
    import hashlib
    import re
    import subprocess
    out = subprocess.run(["ncu", "-i", report, "--page", "raw", "--csv", "--print-units", "base"],
                         capture_output=True, text=True, check=True).stdout
    rows = list(csv.reader(out.splitlines()))
    hdr = rows[0]
    kn, rd, wr = hdr.index("Kernel Name"), hdr.index("dram__bytes_read.sum"), hdr.index("dram__bytes_write.sum")
    pat = re.compile(TRAFFIC_KERNEL_RE[kernel])
    per_launch = []
    for r in rows[1:]:
        if len(r) > max(kn, rd, wr) and pat.search(r[kn]):
            try:
                per_launch.append(int(round(float(r[rd].replace(",", "")) + float(r[wr].replace(",", "")))))
            except ValueError:
                continue   # the units row
    if not per_launch:
        raise SystemExit("no launch of %s in %s" % (kernel, report))
    h = hashlib.sha256()
    for src in TRAFFIC_SOURCES[kernel]:
        with open(os.path.join(ROOT, src), "rb") as f:
            h.update(f.read())
    rec = {"kernel": kernel, "workload": workload, "dram_bytes_per_launch": per_launch,
           "sources": TRAFFIC_SOURCES[kernel], "sha256": h.hexdigest(), "capture": capture_md}
    path = os.path.join(ROOT, "profiles", "traffic_%s_%s.json" % (kernel, workload))
    with open(path, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(path, per_launch)


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return PEAKS_FALLBACK, "fallback"


CLOCK_REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
# throttle reasons that void a timing (sw_power_cap is normal under dense tensor load)
CLOCK_REJECT = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown")


def summarize_clock_lines(lines):
    """Median SM clock, max SM clock and active throttle reasons of nvidia-smi CSV lines
    (`ClockSampler.Q`, noheader, nounits); lines that do not parse are skipped."""
    sm, smax, reasons = [], [], set()
    for ln in lines:
        f = [x.strip() for x in ln.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            smax.append(float(f[2]))
        except ValueError:
            continue
        for nm, v in zip(CLOCK_REASONS, f[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
            "reasons": sorted(reasons), "samples": len(sm)}


def clock_verdict(clk, stuck_frac=0.8):
    """Why a timed region's clock record voids its number, or None: a thermal or hardware
    slowdown was active, or the median SM clock sat below `stuck_frac` of its maximum with
    no reason reported (a clock lock left by another process)."""
    bad = [r for r in clk.get("reasons", []) if r in CLOCK_REJECT]
    if bad:
        return "throttled: " + ",".join(bad)
    sm, smax = clk.get("sm_mhz"), clk.get("sm_max_mhz")
    if sm and smax and sm < stuck_frac * smax and not clk.get("reasons"):
        return "SM clock %.0f of %.0f MHz with no reason reported" % (sm, smax)
    return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region.

    `start()` launches the sampler and waits (up to 5 s) for its first sample, so that
    sampling is live when the timed region begins; only the samples read after that
    point are summarised."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 100

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.first = threading.Event()

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            self.first.wait(timeout=5.0)
            self.lines = []
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())
            self.first.set()

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        # one more period so that the sample covering the end of the region is read
        time.sleep(self.PERIOD_MS / 1000.0)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        return summarize_clock_lines(list(self.lines))


def max_over_ranks(value, world):
    """The largest of every rank's value (the whole job's time), via an all-reduce on the
    process group's device (CUDA tensors for NCCL, host tensors for gloo)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ----------------------------------------------------------------------------- CPU oracle leg
def oracle_sample(wl):
    """The oracle's graph SP2 on a sample workload; returns (orbitals, seconds of gather +
    SP2 + assembly, iterations)."""
    from oracle import graph, hamiltonian, partition, sp2
    w = make_system(wl, wl["seed"])
    thresh, ncell = wl["thresh"], wl["ncell"]
    H = hamiltonian.build_h(w["pos"], w["box"], w["onsite"])
    N = H.shape[0]
    S = graph.h2_threshold(H, thresh)
    subs, nc = partition.subgraphs(S, partition.spatial_cores(w["pos"], w["box"], ncell))
    t0 = time.perf_counter()
    D, log = sp2.sp2_graph(H, subs, nc, N // 2, n_max=48)
    dt = time.perf_counter() - t0
    return N, dt, log.iters


def oracle_full(wl, ncell, gpu_seq):
    """The oracle on the whole workload (cpu_baseline leg): H by the k-d-tree builder, the same
    graph and partition as the GPU run, then graph SP2 with its own FP64 decisions, gather +
    SP2 + assembly timed.  When its branch sequence differs from the GPU run's, the oracle is
    run once more (untimed) replaying the GPU's sequence, so that the D it returns for the
    comparison is the one the GPU computed.  Returns (N, seconds, iterations, D csc, seq
    equal, its own log)."""
    from oracle import graph, hamiltonian, partition, sp2
    w = make_system(wl, wl["seed"])
    H = hamiltonian.build_h_tree(w["pos"], w["box"], w["onsite"])
    N = H.shape[0]
    S = graph.h2_threshold(H, wl["thresh"])
    subs, nc = partition.subgraphs(S, partition.spatial_cores(w["pos"], w["box"], ncell))
    t0 = time.perf_counter()
    D, log = sp2.sp2_graph(H, subs, nc, N // 2, n_max=48)
    dt = time.perf_counter() - t0
    same = list(log.seq) == list(gpu_seq)
    if not same:
        D, _ = sp2.sp2_graph(H, subs, nc, N // 2, seq=list(gpu_seq))
    return N, dt, log.iters, D.tocsc(), same, log


def ell_max_abs_diff(col, val, Dcsc):
    """max |D_gpu - D_ref| over every entry of either (ELL row i = column i of D)."""
    import scipy.sparse as sps
    n, w = col.shape
    m = col >= 0
    cols = np.repeat(np.arange(n), w).reshape(n, w)
    G = sps.csc_matrix((val[m], (col[m], cols[m])), shape=Dcsc.shape)
    diff = (G - Dcsc).tocoo()
    return float(np.abs(diff.data).max()) if diff.nnz else 0.0


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    # each step: the oracle on a 12^3 sample (27 core sets of the 32^3 workload's shape)
    wl = dict(kind="lattice", L=12, seed=0, thresh=0.15, ncell=(3, 3, 3))
    for _ in range(args.warmup):
        oracle_sample(wl)
    ts, its = [], []
    for _ in range(args.steps):
        N, dt, it = oracle_sample(wl)
        ts.append(dt)
        its.append(it)
    value = N * len(ts) / sum(ts)
    sample = "12^3 sample (N=1728, 27 cores of 4^3, |H^2|>=0.15 halos, m_s~430-470) of the 32^3 workload; " \
             "oracle graph SP2 (NumPy FP64), gather+SP2+assembly timed"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * sum(ts) / len(ts),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "lattice32 (oracle on a 12^3 sample)", "iters": its[-1]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- QMD-like run
def configure(args, gbe, ctx, H, parts, prm, X):
    """Launch configuration of the squaring kernel before the timed region: forced by
    --config, the default with --no-autotune, else chosen by the library's autotuner
    (every built configuration timed on this problem, untimed here)."""
    if prm.prec == gbe.PREC_FP64:
        return None
    if args.config:
        v = [int(x) for x in args.config.split(",")]
        gbe.subs_set_config(ctx, X, v[0], v[1], v[2] if len(v) > 2 else 0)
        return {"forced": gbe.subs_get_config(X)}
    if args.no_autotune:
        return {"default": gbe.subs_get_config(X)}
    t0 = time.perf_counter()
    rep = gbe.sp2_autotune(ctx, H, parts, prm, X, reps=3)
    rep["tuning_s"] = time.perf_counter() - t0
    return rep


def run_qmd(args, wl, gbe, torch, dist, ctx, local, rank, world):
    """MD steps of the lattice: every step rebuilds H from the new positions, the graph from
    the previous step's D, the partition, the SP2 state, runs SP2 with the previous step's
    branch sequence replayed, and assembles D (the next step's graph input).  With
    wl["sequence"] == "gap" (Sec. II.C's other source of a sequence) the graph is the
    complete one and each step's sequence comes from the HOMO-LUMO gap estimated from the
    previous step's traces (gbe_sp2_gap_estimate, then gbe_sp2_sequence on the new step's
    Gershgorin bounds).  A step's inputs are the positions, copied in from pinned host
    memory; its output read back is the SP2 report.  Timed: the whole step, wall clock, K
    steps after W warm-up steps."""
    import synth
    prec_name, dtype_name = PRECS[args.prec]
    PREC = getattr(gbe, "PREC_" + prec_name)
    w = make_system(wl, wl["seed"] + rank)
    N = w["pos"].shape[0]
    vel = synth.velocities(N, seed=1 + rank)
    box = w["box"]
    ons = torch.from_numpy(w["onsite"]).cuda()
    pos_h = torch.empty((N, 3), dtype=torch.float64).pin_memory()
    pos_d = torch.empty((N, 3), dtype=torch.float64, device="cuda")
    gap_mode = wl.get("sequence") == "gap"
    full = (gbe.parts_import(ctx, N, np.array([N], np.int32), np.array([0, N], np.int64),
                             np.arange(N, dtype=np.int32)) if wl.get("complete") else None)
    bounds = torch.empty(2, dtype=torch.float64, device="cuda")
    state = {"D": None, "seq": None, "gap": None, "gap_steps": 0, "gap_missed": 0}
    phase = {k: 0.0 for k in ("h_build", "graph", "partition", "sp2_state", "sp2", "assemble")}
    last = {}

    def step(t, timed, free=False):
        def mark(name, t0):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            if timed:
                phase[name] += t1 - t0
            return t1
        t0 = time.perf_counter()
        pos_h.numpy()[:] = synth.advance(w["pos"], vel, box, t)
        pos_d.copy_(pos_h, non_blocking=True)
        st = gbe.sites(pos_d, ons, box)
        Hg = gbe.build_hamiltonian(ctx, st)
        t0 = mark("h_build", t0)
        if full is not None:
            parts = full
        else:
            if state["D"] is None:
                G = gbe.build_graph(ctx, Hg.csr(), gbe.GRAPH_H2_THRESH, thresh=wl["thresh"])
            else:
                G = gbe.build_graph(ctx, Hg.csr(), gbe.GRAPH_D_THRESH, thresh=wl["tau"], D_prev=state["D"])
            t0 = mark("graph", t0)
            parts = gbe.partition(ctx, G, gbe.PART_SPATIAL_CELLS, ncell=wl["ncell"], site_struct=st)
        P, total, max_m = parts.info()
        t0 = mark("partition", t0)
        X = gbe.subs_create(ctx, parts, PREC)
        col = torch.empty((N, max_m), dtype=torch.int32, device="cuda")
        val = torch.empty((N, max_m), dtype=torch.float64, device="cuda")
        t0 = mark("sp2_state", t0)
        if gap_mode and state["gap"] is not None and not free:
            # the sequence that converges the estimated gap on this step's spectral bounds
            gbe.gershgorin_noalloc(ctx, Hg.csr(), bounds)
            eps = tuple(bounds.cpu().tolist())
            seq = gbe.sp2_sequence(eps, state["gap"][0], state["gap"][1], wl["seq_tol"])
            prm = gbe.sp2_params(N / 2.0, prec=PREC, n_max=len(seq), seq=seq, eps=eps)
            used_gap = True
        else:
            seq = None if (gap_mode or free) else state["seq"]
            prm = gbe.sp2_params(N / 2.0, prec=PREC, n_max=64, n_min=10, idem_tol=1e-10, seq=seq,
                                 fp64_tail=args.fp64_tail)
            used_gap = False
        if not timed and "tune" not in last:
            # first warm-up step: tune once; later states of the same shape start with the choice
            last["tune"] = configure(args, gbe, ctx, Hg.csr(), parts, prm, X)
            t0 = time.perf_counter()
        gbe.sp2_run(ctx, Hg.csr(), parts, prm, X)
        rep = gbe.sp2_report_get(ctx, X).as_dict()
        t0 = mark("sp2", t0)
        gbe.assemble_D(ctx, X, parts, col, val)
        mark("assemble", t0)
        if free:
            return col, val
        if gap_mode:
            try:
                state["gap"] = gbe.sp2_gap_estimate(rep, N / 2.0, *wl["gap_window"])
            except gbe.GbeError:
                state["gap_missed"] += int(timed)   # no step in the window: keep the last estimate
            state["gap_steps"] += int(timed and used_gap)
        elif state["seq"] is None:
            state["seq"] = rep["seq"]
        state["D"] = gbe.ell_struct(col, val)
        cc, sptr, _ = parts.export()
        last.update(rep=rep, ms=np.diff(sptr), P=P, cc=cc, col=col, val=val, t=t)

    W = max(args.warmup, 3)
    for t in range(W):
        step(t, False)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    t_start = time.perf_counter()
    for t in range(W, W + args.steps):
        step(t, True)
    torch.cuda.synchronize()
    total = time.perf_counter() - t_start
    clk = clocks.stop()
    total = max_over_ranks(total, world)
    # one more MD step, untimed, launched step by step with CUDA events around every
    # squaring (the timed steps run SP2 as CUDA graphs): the kernel's per-launch time
    ctx.set_profiling(True)
    step(W + args.steps, False)
    ctx.set_profiling(False)
    rep, ms = last["rep"], last["ms"]
    gap_check = None
    if gap_mode:
        # the same positions once more, free running (global traces): the D it converges to
        # against the one the gap-derived sequence gave
        col_f, val_f = step(last["t"], False, free=True)
        gap_check = {"max_abs_dD_vs_free_running": float((val_f - last["val"]).abs().max().item()),
                     "same_pattern": bool(torch.equal(col_f, last["col"]))}
    peaks, peak_kind = load_peaks()
    tc_ms = rep["ms_tc"] / max(1, rep["n_tc"])
    mixed = max(1, rep["iters"] - rep["fp64_iters"])
    achieved = rep["mma_flops"] / mixed / (tc_ms / 1000.0) / 1e12 if tc_ms > 0 else None
    peak = float(peaks["bf16_tflops"])
    value = N * world * args.steps / total
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": W,
        "ms_per_step": 1000.0 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": dtype_name, "data": "synthetic",
        "config": {"workload": args.workload, "N": N, "L": wl["L"], "md_steps_timed": args.steps,
                   "graph": ("complete (one subgraph of every site)" if full is not None else
                             "first step |H^2|>=%g, then |D_prev|>=%g" % (wl["thresh"], wl["tau"])),
                   "branch": ("sequence from the previous step's HOMO-LUMO gap estimate (first step free running)"
                              if gap_mode else "previous step's sequence replayed"), "sp2_iters": rep["iters"],
                   "precision": prec_name, "fp64_tail": args.fp64_tail, "cores": int(last["P"]),
                   "m_s_min": int(ms.min()), "m_s_median": float(np.median(ms)), "m_s_max": int(ms.max()),
                   "l2": "inputs larger than L2 (GB-scale split planes); no flush",
                   "timing": "wall clock over whole MD steps (H build, graph, partition, SP2 state, SP2 as "
                             "CUDA graphs, assembly), positions copied in from pinned host memory each step; "
                             "roofline from one further step launched step by step with CUDA events"},
        "phase_ms_per_step": {k: 1000.0 * v / args.steps for k, v in phase.items()},
        "gap_sequence": None if not gap_mode else {
            "timed_steps_on_a_gap_sequence": state["gap_steps"], "timed_steps_without_estimate": state["gap_missed"],
            "last_gap_estimate_eV": list(state["gap"]) if state["gap"] else None, "window": list(wl["gap_window"]),
            "tol": wl["seq_tol"], **(gap_check or {})},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak if achieved else None, "traffic": None,
                     "kernel": "sp2_square_tc_kernel<%s>" % prec_name,
                     "peak_kind": peak_kind + " dense bf16/fp16 burst", "ms_per_launch": tc_ms},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": N * 24, "d2h_bytes_per_step": 4616},
        "autotune": last.get("tune"),
        "gpu_launches": None,
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- Chebyshev expansion
def run_foe(args, wl, gbe, torch, ctx, local, rank, world):
    """Finite-temperature D by the Chebyshev expansion on the subgraphs (Eq. 7 with Eq. 6):
    one step = gather + order + 1 products + assembly, FP16X6 (timed) and FP64 (one run,
    for max|dD|)."""
    w = make_system(wl, wl["seed"] + rank)
    N = w["pos"].shape[0]
    st = gbe.sites(torch.from_numpy(w["pos"]).cuda(), torch.from_numpy(w["onsite"]).cuda(), w["box"])
    Hh = gbe.build_hamiltonian(ctx, st)
    Hv = Hh.csr()
    G = gbe.build_graph(ctx, Hv, gbe.GRAPH_H2_THRESH, thresh=wl["thresh"])
    parts = gbe.partition(ctx, G, gbe.PART_SPATIAL_CELLS, ncell=wl["ncell"], site_struct=st)
    P, total, max_m = parts.info()
    f = wl["foe"]
    col = {p: torch.empty((N, max_m), dtype=torch.int32, device="cuda") for p in ("m", "d")}
    val = {p: torch.empty((N, max_m), dtype=torch.float64, device="cuda") for p in ("m", "d")}

    def once(X, prec, key):
        rep = gbe.foe_run(ctx, Hv, parts, X, f["beta"], f["mu"], f["order"], prec=prec)
        gbe.assemble_D(ctx, X, parts, col[key], val[key])
        return rep

    Xm = gbe.subs_create(ctx, parts, gbe.PREC_FP16X6)
    for _ in range(max(args.warmup, 3)):
        once(Xm, gbe.PREC_FP16X6, "m")
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        rep = once(Xm, gbe.PREC_FP16X6, "m")
    torch.cuda.synchronize()
    sec = (time.perf_counter() - t0) / args.steps
    clk = clocks.stop()
    sec = max_over_ranks(sec, world)
    Xd = gbe.subs_create(ctx, parts, gbe.PREC_FP64)
    t1 = time.perf_counter()
    repd = once(Xd, gbe.PREC_FP64, "d")
    torch.cuda.synchronize()
    sec_d = time.perf_counter() - t1
    dD = float((val["m"] - val["d"]).abs().max().item()) if torch.equal(col["m"], col["d"]) else float("nan")
    peaks, peak_kind = load_peaks()
    steps = f["order"] + 1
    mma_tflops = rep["mma_flops"] / (rep["ms_steps"] / 1000.0) / 1e12 if rep["ms_steps"] else None
    line = {
        "metric": METRIC, "value": N * world / sec, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": 1000.0 * sec, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f16-split(x6)/f32-acc", "data": "synthetic",
        "config": {"workload": args.workload, "N": N, "L": wl["L"], "graph": "|H^2|>=%g" % wl["thresh"],
                   "cores": int(P), "beta_per_eV": f["beta"], "mu_eV": f["mu"], "order": f["order"],
                   "products_per_D": steps, "scale_B": rep["scale"],
                   "timing": "wall clock per D build (gather, order+1 products, assembly), graph-free host loop"},
        "phase_ms": {"gather": rep["ms_gather"], "products": rep["ms_steps"]},
        "tensor_tflops_in_products": mma_tflops,
        "roofline": {"bound": "tensor", "achieved": mma_tflops, "peak": float(peaks["bf16_tflops"]),
                     "unit": "TFLOP/s", "frac": mma_tflops / float(peaks["bf16_tflops"]) if mma_tflops else None,
                     "traffic": None, "kernel": "sp2_square_tc_kernel<FP16X6, Chebyshev>",
                     "peak_kind": peak_kind + " dense bf16/fp16 burst"},
        "fp64": {"value": N * world / sec_d, "unit": UNIT, "ms_per_step": 1000.0 * sec_d},
        "max_abs_dD_vs_fp64": dD,
        "e2e": {"value": N * world / sec, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": (3 + steps + 2) * args.steps,
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- learned graph proposal
def mlp_init_params(seed):
    """He-normal initial weights of the width-64 network: W1[64x5], b1, W2[64x64], b2, w3, b3."""
    rng = np.random.default_rng(seed)
    return np.concatenate([rng.normal(0.0, (2.0 / 5) ** 0.5, 320), np.zeros(64),
                           rng.normal(0.0, (2.0 / 64) ** 0.5, 4096), np.zeros(64),
                           rng.normal(0.0, (1.0 / 64) ** 0.5, 64), np.zeros(1)]).astype(np.float32)


def mlp_labelled_system(gbe, torch, ctx, cfg, seed, taus):
    """One seeded training system: candidate pairs with features, and for each tau the labels
    |D_ij| >= tau from the library's FP64-grade SP2 on its complete graph (one subgraph of
    every site)."""
    import synth
    n = cfg["train_n"]
    w = synth.disordered(n, seed=seed)
    st = gbe.sites(torch.from_numpy(w["pos"]).cuda(), torch.from_numpy(w["onsite"]).cuda(), w["box"])
    Hh = gbe.build_hamiltonian(ctx, st)
    full = gbe.parts_import(ctx, n, np.array([n], np.int32), np.array([0, n], np.int64), np.arange(n, dtype=np.int32))
    X, rep = gbe.sp2_submatrices(ctx, Hh.csr(), full, gbe.sp2_params(n / 2.0, prec=gbe.PREC_FP64TC, n_max=100))
    col = torch.empty((n, n), dtype=torch.int32, device="cuda")
    val = torch.empty((n, n), dtype=torch.float64, device="cuda")
    gbe.assemble_D(ctx, X, full, col, val)
    P = gbe.pairs_build(ctx, st, Hh.csr(), cfg["rcand"])
    labs = {}
    for tau in taus:
        labs[tau] = torch.empty(P.info()[1], dtype=torch.uint8, device="cuda")
        gbe.mlp_labels(ctx, P, col, val, tau, labs[tau])
    torch.cuda.synchronize()
    return P, labs


def mlp_train(args, gbe, torch, ctx, cfg):
    """Train one network per label threshold on the GPU (the configuration's tau = 1e-5 and
    the pruning threshold cfg["tau"]): args.train_systems labelled systems, one Adam step per
    system in turn, cfg passes; accuracy on an unseen system.  Returns the cfg["tau"]
    network, the 1e-5 one and the training reports."""
    taus = [1e-5, cfg["tau"]] if cfg["tau"] != 1e-5 else [1e-5]
    t0 = time.perf_counter()
    sets = [mlp_labelled_system(gbe, torch, ctx, cfg, cfg["train_seed0"] + k, taus) for k in range(args.train_systems)]
    t_lab = time.perf_counter() - t0
    Pt, labt = mlp_labelled_system(gbe, torch, ctx, cfg, cfg["test_seed"], taus)
    nets, reports = {}, {}
    for tau in taus:
        M = gbe.mlp_create(ctx)
        M.set_params(mlp_init_params(0))
        loss0 = float(np.mean([M.gradient(P, labs[tau])[0] for P, labs in sets]))
        t0 = time.perf_counter()
        for _ in range(cfg["passes"]):
            for P, labs in sets:
                M.train(P, labs[tau], 1, cfg["lr"])
        t_train = time.perf_counter() - t0
        loss = float(np.mean([M.gradient(P, labs[tau])[0] for P, labs in sets]))
        z = torch.empty(Pt.info()[1], dtype=torch.float32, device="cuda")
        M.forward(Pt, z)
        acc = float(((z >= 0) == (labt[tau] > 0)).float().mean())
        pos = float(np.mean([float(labs[tau].float().mean()) for _, labs in sets]))
        nets[tau] = M
        reports["tau=%g" % tau] = {"positive_rate": pos, "loss_initial": loss0, "loss_final": loss,
                                   "unseen_accuracy": acc, "train_s": t_train}
    return nets[cfg["tau"]], nets[1e-5], {
        "systems": len(sets), "system": "%d disordered sites, box %.1fa, seeds %d.." % (
            cfg["train_n"], cfg["train_n"] ** (1.0 / 3.0), cfg["train_seed0"]),
        "labels": "|D_ij| >= tau, D from FP64TC SP2 on the complete graph", "passes": cfg["passes"],
        "lr": cfg["lr"], "labels_s": t_lab, "networks": reports,
        "used_for_the_graphs": "tau=%g (tau = 1e-5 labels almost every candidate, so its network keeps "
                               "nearly the whole ball)" % cfg["tau"]}


def ell_rows_diff(torch, rows, ca, va, cb, vb, n, chunk=8192):
    """(max |A - B|, sum of (A - B)^2, entries) over the union of the entries of the given rows
    of two ELL matrices (row i = column i of D; an entry absent from one side counts as zero
    there)."""
    mx, ss, cnt = 0.0, 0.0, 0
    for r0 in range(0, len(rows), chunk):
        r = rows[r0:r0 + chunk]
        a_c, a_v, b_c, b_v = ca[r], va[r], cb[r], vb[r]
        loc = torch.arange(len(r), device=a_c.device, dtype=torch.int64).unsqueeze(1)
        ma, mb = a_c >= 0, b_c >= 0
        keys = torch.cat([(loc * n + a_c)[ma], (loc * n + b_c)[mb]])
        vals = torch.cat([a_v[ma], -b_v[mb]])
        uk, inv = torch.unique(keys, return_inverse=True)
        d = torch.zeros(len(uk), dtype=torch.float64, device=a_c.device).index_add_(0, inv, vals)
        if len(d):
            mx = max(mx, float(d.abs().max()))
            ss += float((d * d).sum())
            cnt += len(d)
    return mx, ss, cnt


def graph_sp2_batched(gbe, torch, ctx, Hv, parts, N, seq, budget, keep=None, compare=None):
    """FP64-grade graph SP2 (FP64TC) of a partition that need not fit the device at once,
    through gbe_sp2_replay_batched: the subgraphs run in batches whose iterates fit `budget`
    bytes, each replaying the branch sequence `seq` (no traces need to be combined,
    Sec. II.C), and D is assembled column by column.  keep: (col, val) to fill with D;
    compare: {name: (col, val)} D's compared row by row with this one."""
    P, total, max_m = parts.info()
    cc, sptr, _ = parts.export()
    ms = np.diff(sptr)
    need = float(np.sum(((ms + 127) // 128 * 128).astype(np.float64) ** 2)) * 40.0   # 10 planes x 2 B x 2 sides
    col = torch.empty((N, max_m), dtype=torch.int32, device="cuda") if keep is None else keep[0]
    val = torch.empty((N, max_m), dtype=torch.float64, device="cuda") if keep is None else keep[1]
    prm = gbe.sp2_params(N / 2.0, prec=gbe.PREC_FP64TC, n_max=max(len(seq), 10), seq=seq)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    B = gbe.sp2_replay_batched(ctx, Hv, parts, prm, int(budget), col, val)
    torch.cuda.synchronize()
    t_sp2 = time.perf_counter() - t0
    diffs = {}
    rows = torch.arange(N, device="cuda")
    for k, (cb, vb) in (compare or {}).items():
        diffs[k] = list(ell_rows_diff(torch, rows, col, val, cb, vb, N))
    info = {"subgraphs": int(P), "m_s_min": int(ms.min()), "m_s_median": float(np.median(ms)), "m_s_max": int(ms.max()),
            "sum_m3": float(np.sum(ms.astype(np.float64) ** 3)), "batches": B, "planes_gb": need / 1e9,
            "sp2_s": t_sp2, "alg_tflops": 2.0 * float(np.sum(ms.astype(np.float64) ** 3)) * len(seq) / t_sp2 / 1e12}
    return info, diffs


def mlp_compare(args, gbe, torch, ctx, cfg, w, st, Hv, M, M5=None):
    """The trained network's graphs of the big system (one per logit cut) against the H^k
    pattern graphs and the whole candidate ball: each graph's FP64-grade graph SP2 (the
    same replayed branch sequence), D compared with the conservative H^2 graph's D, with
    each graph's sum of m_s^3 and SP2 time."""
    N = w["pos"].shape[0]

    def hk(k):
        return lambda: gbe.build_graph(ctx, Hv, gbe.GRAPH_HK_PATTERN, k=k)

    def learned(cut):
        return lambda: gbe.build_graph(ctx, Hv, gbe.GRAPH_MLP, site_struct=st, mlp=M, rcand=cfg["rcand"],
                                       logit_cut=cut)

    graphs = [("H^1", hk(1))] + [("MLP cut %g" % c, learned(c)) for c in cfg["cuts"]]
    if M5 is not None:
        graphs.append(("MLP tau=1e-5 cut 0", lambda: gbe.build_graph(ctx, Hv, gbe.GRAPH_MLP, site_struct=st, mlp=M5,
                                                                    rcand=cfg["rcand"], logit_cut=0.0)))
    graphs += [("ball r<%g" % cfg["rcand"], learned(-1e30)), ("H^2", hk(2))]
    res, parts_of = {}, {}
    for name, make in graphs:
        t0 = time.perf_counter()
        G = make()
        parts_of[name] = gbe.partition(ctx, G, gbe.PART_SPATIAL_CELLS, ncell=cfg["ncell"], site_struct=st)
        torch.cuda.synchronize()
        res[name] = {"edges_per_site": G.size()[1] / N, "graph_and_partition_s": time.perf_counter() - t0}
        del G
    # the branch sequence: one global-trace run (FP16X6, every subgraph resident: 4 planes x 2
    # bytes x 2 sides per padded element) of the first learned graph, or of H^1 when its
    # planes would not fit beside the rest
    budget = args.batch_gb * 1e9

    def planes16(parts):
        ms = np.diff(parts.export()[1])
        return float(np.sum(((ms + 127) // 128 * 128).astype(np.float64) ** 2)) * 16.0

    first = graphs[1][0]
    src = first if planes16(parts_of[first]) <= 1.5 * budget else "H^1"
    t0 = time.perf_counter()
    XS = gbe.subs_create(ctx, parts_of[src], gbe.PREC_FP16X6)
    gbe.sp2_run(ctx, Hv, parts_of[src], gbe.sp2_params(N / 2.0, prec=gbe.PREC_FP16X6, n_max=cfg["n_max"]), XS)
    rep = gbe.sp2_report_get(ctx, XS).as_dict()
    del XS
    seq = rep["seq"]
    seq_info = {"from": "global-trace FP16X6 run of the %s graph" % src, "steps": len(seq), "stop": rep["stop"],
                "s": time.perf_counter() - t0}
    # the reference first (its D kept), then every other graph compared with it batch by batch
    _, _, max_m = parts_of["H^2"].info()
    ref = (torch.empty((N, max_m), dtype=torch.int32, device="cuda"),
           torch.empty((N, max_m), dtype=torch.float64, device="cuda"))
    info, _ = graph_sp2_batched(gbe, torch, ctx, Hv, parts_of["H^2"], N, seq, budget, keep=ref)
    res["H^2"].update(info)
    for name, _ in graphs[:-1]:
        info, diffs = graph_sp2_batched(gbe, torch, ctx, Hv, parts_of[name], N, seq, budget, compare={"H^2": ref})
        res[name].update(info)
        mx, ss, cnt = diffs["H^2"]
        res[name]["max_abs_dD_vs_H2"] = mx
        res[name]["rms_dD_vs_H2"] = (ss / cnt) ** 0.5 if cnt else 0.0   # over the union of both patterns
        res[name]["sum_m3_vs_H2"] = res[name]["sum_m3"] / res["H^2"]["sum_m3"]
        del parts_of[name]
    return {"graphs": res, "sequence": seq_info, "cores": "spatial cells %s" % (cfg["ncell"],),
            "precision": "FP64TC (FP64-grade tensor-core squarings) in every graph's SP2",
            "reference": "the H^2 pattern graph (every pair with (H^2)_ij != 0)"}


def run_mlp(args, wl, gbe, torch, ctx, local, rank, world):
    """Graph proposal by the edge classifier at full size: per step the candidate pairs and
    their features, the network's logits for every pair, and the selected graph (union
    with H).  Reported: sites/s and pairs/s of the whole proposal; the phases apart.  The
    network is first trained on the GPU (mlp_train); unless --no-compare, the proposed
    graph's FP64-grade SP2 is then compared with the H^k pattern graphs' (mlp_compare)."""
    w = make_system(wl, wl["seed"] + rank)
    N = w["pos"].shape[0]
    st = gbe.sites(torch.from_numpy(w["pos"]).cuda(), torch.from_numpy(w["onsite"]).cuda(), w["box"])
    Hh = gbe.build_hamiltonian(ctx, st)
    Hv = Hh.csr()
    cfg = dict(wl["mlp"])
    if args.mlp_tau is not None:
        cfg["tau"] = args.mlp_tau
    if args.mlp_cuts:
        cfg["cuts"] = tuple(float(c) for c in args.mlp_cuts.split(","))
    M, M5, train = mlp_train(args, gbe, torch, ctx, cfg)
    phases = {"pairs_features": 0.0, "forward": 0.0, "graph": 0.0}
    npairs = 0

    def step(timed):
        nonlocal npairs
        t0 = time.perf_counter()
        P = gbe.pairs_build(ctx, st, Hv, cfg["rcand"])
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        npairs = P.info()[1]
        z = torch.empty(npairs, dtype=torch.float32, device="cuda")
        M.forward(P, z)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        del P, z
        G = gbe.build_graph(ctx, Hv, gbe.GRAPH_MLP, site_struct=st, mlp=M, rcand=cfg["rcand"], logit_cut=cfg["cut"])
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        if timed:
            phases["pairs_features"] += t1 - t0
            phases["forward"] += t2 - t1
            phases["graph"] += t3 - t2
        return G

    for _ in range(max(args.warmup, 3)):
        step(False)
    clocks = ClockSampler(local)
    clocks.start()
    for _ in range(args.steps):
        G = step(True)
    clk = clocks.stop()
    edges = G.size()[1]
    del G
    sec = max_over_ranks(phases["graph"] / args.steps, world)
    fwd = phases["forward"] / args.steps
    flops = 2.0 * npairs * (5 * 64 + 64 * 64 + 64)
    line = {
        "metric": "learned graph proposal: sites/s (candidate pairs, features, network, selection)",
        "value": N * world / sec, "unit": "sites/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": 1000.0 * sec, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f16 tensor-core 64x64 layer (hi+lo activations), f32 accumulation; fp16-rounded weights",
        "data": "synthetic (seeded systems; network trained on the GPU in this run)",
        "config": {"workload": args.workload, "N": N, "box_a": float(w["box"][0]), "rcand_a": cfg["rcand"],
                   "logit_cut": cfg["cut"], "pairs": int(npairs), "graph_edges_per_site": edges / N,
                   "timing": "wall clock of gbe_build_graph(GBE_GRAPH_MLP); pairs and forward timed apart"},
        "phase_ms": {k: 1000.0 * v / args.steps for k, v in phases.items()},
        "pairs_per_s_forward": npairs / fwd,
        "forward_tflops": flops / fwd / 1e12,   # the network's 2 x 4,480 flop per pair; 64x64 layer on mma.sync
        "training": train,
        "e2e": None, "gpu_launches": None, "clocks": clk,
    }
    if not args.no_compare:
        line["comparison"] = mlp_compare(args, gbe, torch, ctx, cfg, w, st, Hv, M, M5)
    if rank == 0:
        print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU leg
def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gbe", choices=["gbe", "reference"])
    ap.add_argument("--workload", default="lattice32", choices=sorted(WORKLOADS))
    ap.add_argument("--fp64-steps", type=int, default=None,
                    help="timed runs of the FP64 path (default 3; 1 on the disordered workloads, ~28 s each)")
    ap.add_argument("--fp64-tail", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--shard", action="store_true",
                    help="with several ranks: one system, its subgraphs dealt to the ranks, the global traces "
                         "all-reduced every SP2 step (strong scaling); default: an independent system per rank")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-fp64tc", action="store_true",
                    help="skip the FP64-grade tensor-core comparison run (default: timed beside the FP64 path)")
    ap.add_argument("--prec", default=None, choices=sorted(PRECS),
                    help="squaring precision (default: fp16x6; fp64tc on the disordered workloads, where "
                         "fp16x6 misses the 1e-6 bound)")
    ap.add_argument("--no-graphs", action="store_true",
                    help="launch SP2 runs step by step instead of as CUDA graphs (profilers do not see "
                         "kernels inside conditional graph nodes)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip the squaring kernel's autotuner (default launch configuration)")
    ap.add_argument("--config", metavar="STAGES,SCHEDULE[,KCHUNK]",
                    help="force the squaring kernel's launch configuration instead of autotuning, e.g. 4,0 "
                         "(schedule 0 round-robin, 1 balanced ranges; K-chunk 32 or 16); used to profile the "
                         "tuned choice")
    ap.add_argument("--train-systems", type=int, default=200,
                    help="mlp1m: seeded 4096-site systems the network is trained on")
    ap.add_argument("--mlp-tau", type=float, default=None,
                    help="mlp workloads: label threshold |D_ij| >= tau (default 1e-2)")
    ap.add_argument("--mlp-cuts", default=None,
                    help="mlp workloads: comma-separated logit cuts of the compared learned graphs")
    ap.add_argument("--no-compare", action="store_true",
                    help="mlp1m: skip the FP64-grade graph SP2 comparison of the proposed graph with H^1 and H^2")
    ap.add_argument("--batch-gb", type=float, default=96.0,
                    help="mlp1m comparison: split-plane bytes per batch of subgraphs (GB)")
    ap.add_argument("--record-traffic", metavar="REPORT",
                    help="write the DRAM traffic record of the FP16X6 squaring kernel for --workload "
                         "from this ncu report (no GPU needed), then exit")
    return ap.parse_args(argv)


def main():
    args = parse_args()
    disordered = WORKLOADS[args.workload]["kind"] == "disordered" and not WORKLOADS[args.workload].get("mlp")
    if args.prec is None:
        args.prec = WORKLOADS[args.workload].get("prec") or ("fp64tc" if disordered else "fp16x6")
    if args.fp64_steps is None:
        args.fp64_steps = 1 if disordered else 3
    if args.record_traffic:
        record_traffic(args.record_traffic, "sp2_square_tc_fp16x6", args.workload,
                       "profiles/sp2_square_tc_%s_%s.md" % (args.prec, args.workload))
        return
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import torch.distributed as dist

    import paper_1603_00937_gb300 as gbe

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    wl = WORKLOADS[args.workload]
    stream = torch.cuda.current_stream().cuda_stream
    ctx = gbe.Context(local, stream)
    ctx.set_graph_launch(not args.no_graphs)
    if wl.get("qmd"):
        run_qmd(args, wl, gbe, torch, dist, ctx, local, rank, world)
        return
    if wl.get("foe"):
        run_foe(args, wl, gbe, torch, ctx, local, rank, world)
        return
    if wl.get("mlp"):
        run_mlp(args, wl, gbe, torch, ctx, local, rank, world)
        return

    # ---------------------------------------------------------------- set-up (timed apart)
    t_setup = time.perf_counter()
    # --shard: one system whose subgraphs are dealt to the ranks (every rank builds the same
    # H, graph and partition); otherwise an independent system per rank
    shard = bool(args.shard) and world > 1
    systems = 1 if shard else world   # systems the ranks process together per step
    w = make_system(wl, wl["seed"] + (0 if shard else rank))
    N = w["pos"].shape[0]
    pos = torch.from_numpy(w["pos"]).cuda()
    ons = torch.from_numpy(w["onsite"]).cuda()
    st = gbe.sites(pos, ons, w["box"])
    Hh = gbe.build_hamiltonian(ctx, st)
    Hv = Hh.csr()
    G = gbe.build_graph(ctx, Hv, gbe.GRAPH_H2_THRESH, thresh=wl["thresh"])
    part_tune = None
    if wl.get("ncell_candidates"):
        prec0 = getattr(gbe, "PREC_" + PRECS[args.prec][0])
        parts, bi, pcost = gbe.partition_autotune(ctx, G, wl["ncell_candidates"], prec=prec0, site_struct=st)
        part_tune = {"candidates": [list(c) for c in wl["ncell_candidates"]],
                     "modelled_squaring_us_per_step": [None if not np.isfinite(c) else float(c) for c in pcost],
                     "chosen": list(wl["ncell_candidates"][bi])}
    else:
        parts = gbe.partition(ctx, G, gbe.PART_SPATIAL_CELLS, ncell=wl["ncell"], site_struct=st)
    P, total, max_m = parts.info()
    cc, sptr, _ = parts.export()
    ms = np.diff(sptr)
    shard_info = None
    if shard:
        owner, load = gbe.shard_assign(sptr, world)
        parts_all = parts
        parts = gbe.parts_shard(ctx, parts_all, owner, rank)
        shard_info = {"ranks": world, "assignment": "greedy longest-processing-time on m_s^3",
                      "subgraphs_per_rank": [int(x) for x in np.bincount(owner, minlength=world)],
                      "load_imbalance": float(load.max() / load.mean()),
                      "exchange": "all-reduce of per-subgraph trace sums (2 P + 1 doubles) after the gather and "
                                  "every SP2 step, NCCL on the context stream"}
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup

    n, width = N, max_m
    col_m = torch.empty((n, width), dtype=torch.int32, device="cuda")
    val_m = torch.empty((n, width), dtype=torch.float64, device="cuda")
    col_d = torch.empty_like(col_m)
    val_d = torch.empty_like(val_m)
    n_max = wl.get("n_max", 48)

    exchange = gbe.dist_exchange() if shard else None

    def params(prec, seq=None):
        return gbe.sp2_params(N / 2.0, prec=prec, n_max=n_max, n_min=10, idem_tol=1e-10,
                              fp64_tail=args.fp64_tail if prec != gbe.PREC_FP64 else 0, seq=seq,
                              exchange=exchange)

    def timed(X, prm, col, val, steps, warmup):
        for _ in range(warmup):
            gbe.sp2_run(ctx, Hv, parts, prm, X)
            gbe.assemble_D(ctx, X, parts, col, val)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            gbe.sp2_run(ctx, Hv, parts, prm, X)
            gbe.assemble_D(ctx, X, parts, col, val)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        ms = max_over_ranks(ms, world)
        return ms, gbe.sp2_report_get(ctx, X).as_dict()

    prec_name, dtype_name = PRECS[args.prec]
    PREC = getattr(gbe, "PREC_" + prec_name)
    Xm = gbe.subs_create(ctx, parts, PREC)
    pm = params(PREC)
    tune = configure(args, gbe, ctx, Hv, parts, pm, Xm)
    clocks = ClockSampler(local)
    clocks.start()
    ms_m, rep_m = timed(Xm, pm, col_m, val_m, args.steps, max(args.warmup, 3))
    clk = clocks.stop()
    why = clock_verdict(clk)
    # the D of the timed (free-running) build, for the comparison with the oracle
    D_timed = (col_m.cpu().numpy(), val_m.cpu().numpy()) if rank == 0 and world == 1 and \
        not args.no_cpu_baseline and wl["kind"] == "lattice" else None
    # a throttled or clock-locked run is measured once more, on every rank if on any
    if max_over_ranks(1.0 if why else 0.0, world) > 0:
        first = {"ms_per_step": ms_m, "clocks": clk, "why": why or "another rank's clocks"}
        clocks = ClockSampler(local)
        clocks.start()
        ms_m, rep_m = timed(Xm, pm, col_m, val_m, args.steps, max(args.warmup, 3))
        clk = dict(clocks.stop(), remeasured=first)
    # per-launch timing of the squaring kernel: the same run launched step by step with CUDA
    # events around every squaring (the timed runs above are graph-launched)
    ctx.set_profiling(True)
    for _ in range(2):
        gbe.sp2_run(ctx, Hv, parts, pm, Xm)
    rep_prof = gbe.sp2_report_get(ctx, Xm).as_dict()
    ctx.set_profiling(False)

    out = {}
    if not args.no_fp64:
        Xd = gbe.subs_create(ctx, parts, gbe.PREC_FP64)
        ms_d, rep_d = timed(Xd, params(gbe.PREC_FP64), col_d, val_d, args.fp64_steps, 1)
        seq_equal = rep_d["seq"] == rep_m["seq"]
        dD_free = float((val_m - val_d).abs().max().item()) if torch.equal(col_m, col_d) else float("nan")
        # same branch sequence for the precision comparison: replay the FP64 run's sequence
        gbe.sp2_run(ctx, Hv, parts, params(PREC, seq=rep_d["seq"]), Xm)
        gbe.assemble_D(ctx, Xm, parts, col_m, val_m)
        torch.cuda.synchronize()
        dD = float((val_m - val_d).abs().max().item())
        out["fp64"] = {"value": N * systems / (ms_d / 1000.0), "unit": UNIT, "ms_per_step": ms_d,
                       "steps": args.fp64_steps, "iters": rep_d["iters"], "stop": rep_d["stop"],
                       # graph-launched: no per-kernel events, the SP2 phase is the FP64 squarings
                       "fp64_tflops_executed": rep_d["fp64_flops"] / ((rep_d["ms_fp64"] or rep_d["ms_sp2"]) / 1000.0)
                       / 1e12 if (rep_d["ms_fp64"] or rep_d["ms_sp2"]) else None,
                       "alg_tflops": rep_d["alg_flops"] / (ms_d / 1000.0) / 1e12}
        out["max_abs_dD_vs_fp64"] = dD
        out["max_abs_dD_vs_fp64_free_running"] = dD_free
        out["branch_sequences_equal"] = seq_equal
        # the metric compares mixed with FP64 at max|dD| <= 1e-6: a mixed result outside that
        # gate is marked and takes no part in a speedup
        out["within_1e-6_gate"] = bool(dD <= 1e-6)
        if dD <= 1e-6:
            out["speedup_vs_fp64"] = ms_d / ms_m
        else:
            out["speedup_vs_fp64"] = None
            out["out_of_tolerance"] = "max|dD| = %.3g against the FP64 path exceeds the metric's 1e-6" % dD
        if PREC != gbe.PREC_FP64TC and not args.no_fp64tc:
            # the FP64-grade tensor-core path on the same workload and sequence as the FP64 run
            Xt = gbe.subs_create(ctx, parts, gbe.PREC_FP64TC)
            col_t, val_t = torch.empty_like(col_m), torch.empty_like(val_m)
            pt = params(gbe.PREC_FP64TC, seq=rep_d["seq"])
            ms_t, rep_t = timed(Xt, pt, col_t, val_t, max(3, args.fp64_steps), 3)
            ctx.set_profiling(True)
            gbe.sp2_run(ctx, Hv, parts, pt, Xt)
            rep_tp = gbe.sp2_report_get(ctx, Xt).as_dict()
            ctx.set_profiling(False)
            tl = rep_tp["ms_tc"] / max(1, rep_tp["n_tc"])
            dT = float((val_t - val_d).abs().max().item())
            out["fp64tc"] = {"value": N * systems / (ms_t / 1000.0), "unit": UNIT, "ms_per_step": ms_t,
                             "iters": rep_t["iters"], "max_abs_dD_vs_fp64": dT,
                             "speedup_vs_fp64": ms_d / ms_t if dT <= 1e-6 else None, "ms_per_squaring_launch": tl,
                             "alg_tflops_in_squarings": rep_tp["alg_flops"] / max(1, rep_tp["iters"]) / (tl / 1000.0) / 1e12
                             if tl > 0 else None,
                             "precision": "FP64TC: five fixed-point fp16 slices, 18 products, FP32 accumulators"}
            del Xt, col_t, val_t

    # ---------------------------------------------------------------- end to end (host buffers)
    def dev_to_host(ptr, count, typestr):
        class _A:
            pass
        a = _A()
        a.__cuda_array_interface__ = {"shape": (int(count),), "typestr": typestr, "data": (int(ptr), False),
                                      "version": 3}
        return torch.as_tensor(a, device="cuda").cpu()

    rp_h = dev_to_host(Hv.rowptr, N + 1, "<i8").pin_memory()
    ci_h = dev_to_host(Hv.col, Hv.nnz, "<i4").pin_memory()
    va_h = dev_to_host(Hv.val, Hv.nnz, "<f8").pin_memory()
    Hhost = gbe.csr(N, rp_h.numpy(), ci_h.numpy(), va_h.numpy())
    col_h = torch.empty((n, width), dtype=torch.int32).pin_memory()
    val_h = torch.empty((n, width), dtype=torch.float64).pin_memory()
    for _ in range(max(args.warmup, 3)):
        gbe.sp2_submatrices(ctx, Hhost, parts, pm, Xm)
        gbe.assemble_D(ctx, Xm, parts, col_h.numpy(), val_h.numpy())
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    e2e_steps = max(1, args.steps)
    for _ in range(e2e_steps):
        gbe.sp2_submatrices(ctx, Hhost, parts, pm, Xm)
        gbe.assemble_D(ctx, Xm, parts, col_h.numpy(), val_h.numpy())
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_s = max_over_ranks(e2e_s, world)
    h2d = (N + 1) * 8 + Hv.nnz * 12
    d2h = n * width * 12 + 4616

    # ---------------------------------------------------------------- roofline of the squaring kernel
    peaks, peak_kind = load_peaks()
    tc_ms = rep_prof["ms_tc"] / max(1, rep_prof["n_tc"])
    mixed_prof = max(1, rep_prof["iters"] - rep_prof["fp64_iters"])
    tc_flops = rep_prof["mma_flops"] / mixed_prof          # executed split-product MMA flops per launch
    alg_flops = rep_prof["alg_flops"] / max(1, rep_prof["iters"])   # sum_s 2 m_s^3 per launch
    achieved_exec = tc_flops / (tc_ms / 1000.0) / 1e12 if tc_ms > 0 else None
    achieved = alg_flops / (tc_ms / 1000.0) / 1e12 if tc_ms > 0 else None
    peak = float(peaks["bf16_tflops"])
    traffic = captured_traffic("sp2_square_tc_fp16x6", args.workload) if prec_name == "FP16X6" else None
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if achieved else None, "traffic": traffic,
                "traffic_unit": "bytes per launch (ncu dram read+write)",
                "work": "algorithmic: sum over subgraphs of 2 m_s^3 per launch (%.4g flop)" % alg_flops,
                "frac_alg": achieved / peak if achieved else None,
                "achieved_exec": achieved_exec, "frac_exec": achieved_exec / peak if achieved_exec else None,
                "work_exec": "executed: %d split products on the padded upper 128x128 tiles (%.4g flop per launch)"
                             % ({"FP16X6": 6, "BF16X3": 3, "FP64TC": 18}[prec_name], tc_flops),
                "kernel": "sp2_square_tc_kernel<%s>" % prec_name, "peak_kind": peak_kind + " dense bf16/fp16 burst",
                "launches": rep_prof["n_tc"], "ms_per_launch": tc_ms,
                "timing": "CUDA events around every squaring of a step-by-step launched run of the same workload"}

    mixed_iters = rep_m["iters"] - rep_m["fp64_iters"]
    # graph-launched run: init, bounds, gather, decision, then per step a squaring and its
    # decision (two more per step with an FP64 tail), then ELL fill and assembly
    launches = 4 + rep_m["iters"] * (2 + (2 if args.fp64_tail > 0 else 0)) + 2
    tiles = [(int(m) + 127) // 128 for m in ms]
    plane_gb = 2 * (4 if prec_name == "FP16X6" else 2) * 2 * 128 * 128 * sum(t * (t + 1) // 2 for t in tiles) / 1e9
    geometry = {"L": wl["L"]} if wl["kind"] == "lattice" else {"box_a": float(w["box"][0])}
    line = {
        "metric": METRIC, "value": N * systems / (ms_m / 1000.0), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms_m, "higher_is_better": True,
        "scaling": "strong" if shard else "weak", "vs_baseline": None, "dtype": dtype_name, "data": "synthetic",
        "config": {"workload": args.workload, "N": N, **geometry, "graph": "|H^2|>=%g" % wl["thresh"],
                   "cores": int(P), "core_size": int(np.median(cc)), "m_s_min": int(ms.min()),
                   "m_s_median": float(np.median(ms)), "m_s_max": int(ms.max()), "precision": prec_name,
                   "fp64_tail": args.fp64_tail, "branch": "global FP64 trace on device, stall stop",
                   "iters": rep_m["iters"], "stop": rep_m["stop"],
                   "l2": "inputs larger than L2: %.2f GB of split planes (2 sides, upper 128-blocks) vs 129 MB "
                         "L2; no flush" % plane_gb,
                   "setup_s": setup_s,
                   "parallelism": ("one system sharded over %d GPUs" % world) if shard else
                                  ("independent system per GPU" if world > 1 else "1 GPU"),
                   "graph_note": ("|H^2| threshold knob in place of the stated |D|>=1e-5 graph: on this model "
                                  "|D|>=1e-5 reaches ~14a, so the literal graph gives m_s ~ N; the knob gives the "
                                  "stated m_s range") if wl["kind"] == "lattice" else
                                 ("|H^2| threshold knob: the near-metallic model has no locality at |D|>=1e-5")},
        "accuracy": {"idem_err_final": rep_m["idem_err"], "trace_minus_n_occ": rep_m["trace"] - N / 2.0,
                     "note": "e_n = |Tr X - Tr X^2| over core positions of the final iterate (stall stop on a "
                             "truncated graph); max|dD| against the FP64 GPU path and the oracle below"},
        "tensor_tflops": rep_m["mma_flops"] / (ms_m / 1000.0) / 1e12,
        "tensor_tflops_in_squarings": achieved,
        "alg_tflops": rep_m["alg_flops"] / (ms_m / 1000.0) / 1e12,
        "phase_ms": {"gather": rep_m["ms_gather"], "sp2": rep_m["ms_sp2"], "squarings": rep_prof["ms_tc"]},
        "roofline": roofline,
        "e2e": {"value": N * systems / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches * args.steps,
        "clocks": clk,
        "autotune": tune,
    }
    if part_tune:
        line["partition_autotune"] = part_tune
    if shard_info:
        line["shard"] = shard_info
    line.update(out)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        if wl["kind"] == "lattice":
            # the whole workload: same graph, same partition, the oracle's own decisions
            ncell = tuple(part_tune["chosen"]) if part_tune else wl["ncell"]
            Ns, dt, it, Dref, same, olog = oracle_full(wl, ncell, rep_m["seq"])
            dD_or = ell_max_abs_diff(D_timed[0], D_timed[1], Dref)
            line["cpu_baseline"] = {
                "value": Ns / dt, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                "sample": "the whole %s workload (N=%d, the GPU run's graph and %d cores), oracle graph SP2 "
                          "(NumPy FP64, %d iterations, %s stop), gather+SP2+assembly timed (%.1f s)"
                          % (args.workload, Ns, int(P), it, olog.stop, dt),
                "branch_sequence_equal_to_gpu": same}
            line["accuracy"]["max_abs_dD_vs_oracle"] = dD_or
            line["accuracy"]["oracle_compared"] = ("oracle's own run (same branch sequence as the GPU's)" if same
                                                   else "oracle replaying the GPU run's branch sequence")
        else:
            swl = WORKLOADS["disordered4k"]
            what = "4096-site sample of the same disordered model (box 16a, 64 cells, |H^2|>=0.1 halos)"
            Ns, dt, it = oracle_sample(swl)
            line["cpu_baseline"] = {"value": Ns / dt, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                                    "sample": what + ", oracle graph SP2 (NumPy FP64, %d iterations), "
                                              "gather+SP2+assembly timed (%.1f s)" % (it, dt)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
