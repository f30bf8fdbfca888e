"""GPU tests of the squaring kernel's launch configurations and of the autotuner.

Workload: the 4096-site sample of the disordered model (box 16a, 4x4x4 spatial-cell
cores, |H^2| >= 0.1): 64 subgraphs of uneven size spread over several 128-wide buckets,
so one launch holds ~1000 upper tiles of different K depths, several per CTA, with
ragged edges.  The oracle's free-running branch sequence is replayed on the GPU.

(a) Every built configuration (K-chunk width x ring depth x tile schedule) gives bit-identical
    D and traces: a tile is computed by the same instructions in the same order
    whichever CTA runs it, and the per-tile trace partials are summed in tile order.
(b) The autotuner times every configuration, installs the fastest, and caches it by
    state shape: a new state of the same shape starts with it, and tuning that state
    again returns the cached choice without timing.  The tuned run matches the oracle
    within the mixed-precision bound of this model (1e-5 for FP16X6).
(c) A depth the kernel is not built with, or an unknown schedule, is rejected.
"""
import numpy as np
import pytest

import synth
from oracle import graph, hamiltonian, partition, sp2

pytestmark = pytest.mark.gpu

from tests.gpu_helpers import assembled_dense, device_csr, gbe, import_parts, torch  # noqa: E402,F401

# ring depths each precision is built with, per K-chunk width
STAGES = {gbe.PREC_FP16X6: {32: [3, 4], 16: [6, 8]}, gbe.PREC_BF16X3: {32: [4, 6, 7], 16: [12, 14]},
          gbe.PREC_FP64TC: {16: [3]}}
N = 4096


@pytest.fixture(scope="module")
def ctx():
    return gbe.Context(0)


@pytest.fixture(scope="module")
def case():
    w = synth.disordered(N, seed=0)
    H = hamiltonian.build_h(w["pos"], w["box"], w["onsite"])
    S = graph.h2_threshold(H, 0.1)
    subs, nc = partition.subgraphs(S, partition.spatial_cores(w["pos"], w["box"], (4, 4, 4)))
    D, log = sp2.sp2_graph(H, subs, nc, N // 2, n_max=60)
    return dict(H=H, subs=subs, nc=nc, D=D.toarray(), seq=log.seq)


def run(ctx, Hd, parts, params, X):
    gbe.sp2_run(ctx, Hd, parts, params, X)
    rep = gbe.sp2_report_get(ctx, X).as_dict()
    assert rep["status"] == 0 and rep["iters"] == params.seq_len
    D, _, _ = assembled_dense(ctx, X, parts, N)
    return D, rep


@pytest.mark.parametrize("prec", [gbe.PREC_FP16X6, gbe.PREC_BF16X3, gbe.PREC_FP64TC])
def test_every_config_gives_identical_D(ctx, case, prec):
    parts = import_parts(ctx, N, case["subs"], case["nc"])
    Hd = device_csr(case["H"])
    params = gbe.sp2_params(N // 2, prec=prec, seq=case["seq"])
    X = gbe.subs_create(ctx, parts, prec)
    ms = np.array([len(s) for s in case["subs"]])
    assert len(np.unique((ms + 127) // 128)) >= 2
    assert gbe.subs_get_config(X) == dict(stages=0, schedule=gbe.SCHED_ROUND_ROBIN, kchunk=0)
    D0, rep0 = run(ctx, Hd, parts, params, X)
    for kc, depths in STAGES[prec].items():
        for stages in depths:
            for sched in (gbe.SCHED_ROUND_ROBIN, gbe.SCHED_BALANCED_RANGES):
                gbe.subs_set_config(ctx, X, stages, sched, kc)
                assert gbe.subs_get_config(X) == dict(stages=stages, schedule=sched, kchunk=kc)
                D, rep = run(ctx, Hd, parts, params, X)
                assert np.array_equal(D, D0), (kc, stages, sched, np.abs(D - D0).max())
                assert rep["t1"] == rep0["t1"] and rep["t2"] == rep0["t2"], (kc, stages, sched)
    if prec in (gbe.PREC_FP16X6, gbe.PREC_FP64TC):
        err = np.abs(D0 - case["D"]).max()
        print(f"disordered 4096, prec {prec}: max|dD| {err:.3e}")
        # the mixed and FP64-grade bounds of this near-metallic sample (test_gpu_disordered.py)
        assert err <= (1e-5 if prec == gbe.PREC_FP16X6 else 5e-10), err


def test_autotune_installs_fastest_and_caches(case):
    ctx = gbe.Context(0)   # empty tuning cache
    parts = import_parts(ctx, N, case["subs"], case["nc"])
    Hd = device_csr(case["H"])
    params = gbe.sp2_params(N // 2, prec=gbe.PREC_FP16X6, seq=case["seq"])
    X = gbe.subs_create(ctx, parts, gbe.PREC_FP16X6)
    D0, _ = run(ctx, Hd, parts, params, X)
    rep = gbe.sp2_autotune(ctx, Hd, parts, params, X, reps=2)
    print("autotune:", rep)
    cands = rep["candidates"]
    assert not rep["cached"] and rep["iters"] == len(case["seq"])
    want = {(kc, s, n) for kc, depths in STAGES[gbe.PREC_FP16X6].items() for s in depths
            for n in ("round_robin", "balanced_ranges")}
    assert len(cands) == len(want)
    assert {(c["kchunk"], c["stages"], c["schedule"]) for c in cands} == want
    assert all(c["ms_per_run"] > 0 for c in cands)
    best = rep["best"]
    assert best["ms_per_run"] == min(c["ms_per_run"] for c in cands)
    cfg = gbe.subs_get_config(X)
    assert cfg["stages"] == best["stages"] and gbe.SCHED_NAMES[cfg["schedule"]] == best["schedule"]
    assert (cfg["kchunk"] or 32) == best["kchunk"]
    D, _ = run(ctx, Hd, parts, params, X)
    assert np.array_equal(D, D0)
    assert np.abs(D - case["D"]).max() <= 1e-5
    # a new state of the same shape starts with the tuned configuration
    X2 = gbe.subs_create(ctx, parts, gbe.PREC_FP16X6)
    assert gbe.subs_get_config(X2) == cfg
    rep2 = gbe.sp2_autotune(ctx, Hd, parts, params, X2, reps=2)
    assert rep2["cached"] and len(rep2["candidates"]) == 1
    D2, _ = run(ctx, Hd, parts, params, X2)
    assert np.array_equal(D2, D0)
    # a state of another precision has its own entry
    X3 = gbe.subs_create(ctx, parts, gbe.PREC_BF16X3)
    assert gbe.subs_get_config(X3) == dict(stages=0, schedule=gbe.SCHED_ROUND_ROBIN, kchunk=0)
    for h in (X3, X2, X, parts):
        h.close()
    ctx.close()


def test_invalid_config_rejected(ctx, case):
    parts = import_parts(ctx, N, case["subs"], case["nc"])
    X = gbe.subs_create(ctx, parts, gbe.PREC_FP16X6)
    for stages, sched, kc in ((5, 0, 0), (6, 0, 32), (4, 0, 16), (4, 7, 0), (-1, 0, 0), (4, 0, 8)):
        with pytest.raises(gbe.GbeError) as e:
            gbe.subs_set_config(ctx, X, stages, sched, kc)
        assert e.value.code == gbe.GBE_EINVAL
    assert gbe.subs_get_config(X) == dict(stages=0, schedule=gbe.SCHED_ROUND_ROBIN, kchunk=0)
