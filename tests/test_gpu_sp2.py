"""GPU parity of the SP2 core (gather, squarings, traces/branch, assembly) against the oracle.

Partitions come from the oracle and enter libgbe through gbe_parts_import, so these tests
isolate the SP2 kernels; the graph and partition kernels have their own parity tests.
Tolerances: FP64 path and the FP64-grade tensor-core path (FP64TC) 1e-10 (max |dD| against
the FP64 oracle on the same graph and branch sequence); FP16X6 tensor-core path 1e-6;
BF16X3 reported, bounded loosely.
"""
import numpy as np
import pytest

from oracle import graph, partition, sp2

pytestmark = pytest.mark.gpu

from tests.gpu_helpers import (assembled_dense, device_csr, gbe, host_csr, import_parts,  # noqa: E402
                               lattice_case, oracle_graph_sp2, torch)


@pytest.fixture(scope="module")
def ctx():
    return gbe.Context(0)


@pytest.fixture(scope="module")
def c1():
    w, H, S, subs, nc = lattice_case(8, seed=0, thr=1e-5)
    N = H.shape[0]
    _, logd = sp2.sp2_dense(H, N // 2)
    Dref, logr, xs = oracle_graph_sp2(H, subs, nc, seq=logd.seq)
    return dict(w=w, H=H, subs=subs, nc=nc, seq=logd.seq, Dref=Dref, logr=logr)


def run(ctx, case, prec, seq=None, **kw):
    H = case["H"]
    N = H.shape[0]
    parts = import_parts(ctx, N, case["subs"], case["nc"])
    p = gbe.sp2_params(N // 2, prec=prec, seq=seq, **kw)
    X, rep = gbe.sp2_submatrices(ctx, device_csr(H), parts, p)
    D, col, val = assembled_dense(ctx, X, parts, N)
    return D, rep, parts, X


def test_fp64_replay_parity(ctx, c1):
    D, rep, _, _ = run(ctx, c1, gbe.PREC_FP64, seq=c1["seq"])
    assert rep["iters"] == len(c1["seq"]) and rep["stop"] == "replay"
    err = np.abs(D - c1["Dref"]).max()
    assert err <= 1e-10, err
    # traces recorded on the device follow the oracle's FP64 traces
    np.testing.assert_allclose(rep["t1"], c1["logr"].t1, rtol=0, atol=1e-9)
    np.testing.assert_allclose(rep["t2"], c1["logr"].t2, rtol=0, atol=1e-9)
    lo, hi = sp2.gershgorin(c1["H"])
    assert abs(rep["eps"][0] - lo) < 1e-12 and abs(rep["eps"][1] - hi) < 1e-12


@pytest.mark.parametrize("prec", [gbe.PREC_FP64, gbe.PREC_FP64TC])
def test_fp64_free_running_matches_oracle_decisions(ctx, c1, prec):
    H = c1["H"]
    N = H.shape[0]
    _, logo, _ = oracle_graph_sp2(H, c1["subs"], c1["nc"], seq=None)
    _, rep, _, _ = run(ctx, c1, prec, seq=None, n_max=60)
    assert rep["stop"] == logo.stop
    assert rep["seq"] == logo.seq


def test_fp64tc_replay_parity(ctx, c1):
    """The FP64-grade tensor-core squaring (five fixed-point fp16 slices, 18 products in four
    FP32 accumulators, the three leading ones exact) against the FP64 oracle."""
    D, rep, _, _ = run(ctx, c1, gbe.PREC_FP64TC, seq=c1["seq"])
    assert rep["iters"] == len(c1["seq"]) and rep["stop"] == "replay" and rep["fp64_iters"] == 0
    err = np.abs(D - c1["Dref"]).max()
    print(f"FP64TC 8^3: {rep['iters']} steps, max|dD| {err:.3e}")
    assert err <= 1e-10, err
    np.testing.assert_allclose(rep["t1"], c1["logr"].t1, rtol=0, atol=1e-9)
    np.testing.assert_allclose(rep["t2"], c1["logr"].t2, rtol=0, atol=1e-9)


def test_fp64_host_csr_e2e(ctx, c1):
    H = c1["H"]
    N = H.shape[0]
    parts = import_parts(ctx, N, c1["subs"], c1["nc"])
    p = gbe.sp2_params(N // 2, prec=gbe.PREC_FP64, seq=c1["seq"])
    X, rep = gbe.sp2_submatrices(ctx, host_csr(H), parts, p)
    n, width = gbe.assemble_width(ctx, X, parts)
    col = np.zeros((n, width), dtype=np.int32)
    val = np.zeros((n, width), dtype=np.float64)
    gbe.assemble_D(ctx, X, parts, col, val)
    D = gbe.ell_to_dense(col, val, N)
    assert np.abs(D - c1["Dref"]).max() <= 1e-10


@pytest.mark.parametrize("tail", [0, 2])
def test_fp16x6_replay_parity(ctx, c1, tail):
    D, rep, _, _ = run(ctx, c1, gbe.PREC_FP16X6, seq=c1["seq"], fp64_tail=tail)
    assert rep["iters"] == len(c1["seq"]) and rep["fp64_iters"] == tail
    err = np.abs(D - c1["Dref"]).max()
    assert err <= 1e-6, err


def test_bf16x3_replay_bounded(ctx, c1):
    D, rep, _, _ = run(ctx, c1, gbe.PREC_BF16X3, seq=c1["seq"])
    err = np.abs(D - c1["Dref"]).max()
    assert err <= 1e-3, err


@pytest.mark.parametrize("prec,tol", [(0, 1e-13), (1, 3e-9), (2, 3e-4), (3, 1e-13)])
@pytest.mark.parametrize("b", [1, 0])
def test_single_step(ctx, c1, prec, tol, b):
    """One squaring X_1 = X_0^2 (b=1) or 2 X_0 - X_0^2 (b=0): dense per-subgraph check."""
    H = c1["H"]
    N = H.shape[0]
    D, rep, parts, X = run(ctx, c1, prec, seq=[b])
    _, _, xs = oracle_graph_sp2(H, c1["subs"], c1["nc"], seq=[b])
    for s in (0, 17, 63):
        m = len(c1["subs"][s])
        got = X.export(s, m)
        assert np.abs(got - xs[s]).max() <= tol
        if prec == gbe.PREC_FP64:
            np.testing.assert_array_equal(got, got.T)  # same products, same order: exact
        else:
            # off-diagonal tiles are mirrored (exact); inside diagonal tiles (a,b) and (b,a)
            # accumulate their split products in different orders
            sym = {gbe.PREC_FP16X6: 1e-9, gbe.PREC_BF16X3: 1e-7, gbe.PREC_FP64TC: 1e-14}[prec]
            assert np.abs(got - got.T).max() <= sym


def ragged_case(seed=3, thr=0.3):
    """Uneven subgraphs (m not multiples of 128, several tiles, small ones) on an 8^3 lattice."""
    import synth
    from oracle import hamiltonian
    w = synth.lattice(8, seed=seed)
    H = hamiltonian.build_h(w["pos"], w["box"], w["onsite"])
    S = graph.h2_threshold(H, thr)
    N = H.shape[0]
    rng = np.random.default_rng(seed)
    perm = rng.permutation(N)
    sizes = [1, 3, 37, 64, 150, 2]
    cores, k = [], 0
    while k < N:
        sz = sizes[len(cores) % len(sizes)]
        cores.append(np.sort(perm[k:k + sz]))
        k += sz
    subs, nc = partition.subgraphs(S, cores)
    return dict(H=H, subs=subs, nc=nc)


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-6), (3, 1e-10)])
def test_ragged_subgraphs(ctx, prec, tol):
    case = ragged_case()
    H = case["H"]
    N = H.shape[0]
    _, logd = sp2.sp2_dense(H, N // 2)
    Dref, _, _ = oracle_graph_sp2(H, case["subs"], case["nc"], seq=logd.seq)
    ms = [len(s) for s in case["subs"]]
    assert max(ms) > 256 and min(ms) < 100 and any(c > 128 for c in case["nc"])
    D, rep, _, _ = run(ctx, case, prec, seq=logd.seq)
    assert np.abs(D - Dref).max() <= tol


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-6), (3, 1e-10)])
def test_tiny_subgraphs(ctx, prec, tol):
    """Very sparse graph: subgraphs of fewer than 32 vertices (a single K-chunk)."""
    case = ragged_case(seed=5, thr=1.5)
    H = case["H"]
    _, logd = sp2.sp2_dense(H, H.shape[0] // 2)
    Dref, _, _ = oracle_graph_sp2(H, case["subs"], case["nc"], seq=logd.seq)
    assert min(len(s) for s in case["subs"]) < 32
    D, rep, _, _ = run(ctx, case, prec, seq=logd.seq)
    assert np.abs(D - Dref).max() <= tol


@pytest.mark.parametrize("prec", [gbe.PREC_FP64, gbe.PREC_FP64TC])
def test_complete_graph_matches_eigh(ctx, prec):
    """One subgraph covering everything: graph SP2 is dense SP2, which is theta(mu - H)."""
    from oracle import exact
    w, H, _, _, _ = lattice_case(6, seed=4)
    N = H.shape[0]
    case = dict(H=H, subs=[np.arange(N)], nc=np.array([N]))
    Dex, _ = exact.density_matrix(H, N // 2)
    D, rep, _, _ = run(ctx, case, prec, n_max=80, idem_tol=1e-11)
    assert rep["stop"] == "tol"
    assert np.abs(D - Dex).max() <= 1e-10


def test_drop_tolerance_and_width_query(ctx, c1):
    H = c1["H"]
    N = H.shape[0]
    _, rep, parts, X = run(ctx, c1, gbe.PREC_FP64, seq=c1["seq"])
    D0, col0, _ = assembled_dense(ctx, X, parts, N)
    D1, col1, val1 = assembled_dense(ctx, X, parts, N, drop_tol=1e-3)
    ref = np.where(np.abs(c1["Dref"]) >= 1e-3, c1["Dref"], 0.0)
    assert np.abs(D1 - ref).max() <= 1e-10
    assert (col1 >= 0).sum() < (col0 >= 0).sum()
    # packed rows: padding only after the kept entries
    for r in range(0, N, 51):
        k = (col1[r] >= 0).sum()
        assert np.all(col1[r, :k] >= 0) and np.all(col1[r, k:] == -1)


@pytest.mark.parametrize("prec", [gbe.PREC_FP64, gbe.PREC_FP16X6, gbe.PREC_FP64TC])
def test_graph_launch_matches_step_launch(prec):
    """The CUDA-graph path (device-driven loop) and the step-by-step launch path run the same
    kernels: identical decisions and bit-identical D.  A state's first run with given inputs
    and parameters is launched step by step, the second captures the graphs, later ones
    relaunch them; a change of parameters goes back to a step-by-step run."""
    case = ragged_case()
    H = case["H"]
    N = H.shape[0]
    outs = []
    for mode in ("graph", "steps", "profiled", "graph-again"):
        ctx = gbe.Context(0)
        ctx.set_graph_launch(mode != "steps")
        ctx.set_profiling(mode == "profiled")
        parts = import_parts(ctx, N, case["subs"], case["nc"])
        Hd = device_csr(H)
        p = gbe.sp2_params(N // 2, prec=prec, n_max=60)
        X, rep = gbe.sp2_submatrices(ctx, Hd, parts, p)
        if mode != "steps":
            X, rep = gbe.sp2_submatrices(ctx, Hd, parts, p, X)          # captured (graph modes)
        if mode == "graph-again":
            X, rep = gbe.sp2_submatrices(ctx, Hd, parts, p, X)          # relaunched
            short = gbe.sp2_params(N // 2, prec=prec, seq=rep["seq"][:5])
            for _ in range(2):                                           # new parameters: steps, capture
                X2, rep2 = gbe.sp2_submatrices(ctx, Hd, parts, short, X)
                assert rep2["iters"] == 5
            for _ in range(2):                                           # back: steps, capture
                X, rep = gbe.sp2_submatrices(ctx, Hd, parts, p, X)
        D, _, _ = assembled_dense(ctx, X, parts, N)
        outs.append((rep["seq"], rep["stop"], D))
    for seq, stop, D in outs[1:]:
        assert seq == outs[0][0] and stop == outs[0][1]
        np.testing.assert_array_equal(D, outs[0][2])


@pytest.mark.parametrize("cover", [True, False])
def test_assembly_into_host_buffers(ctx, c1, cover):
    """Device buffers, page-locked host buffers and pageable host arrays receive the same ELL
    D, every entry written; with cores that leave vertices out (no padding pass can be
    skipped then), those rows stay empty in all three."""
    H = c1["H"]
    N = H.shape[0]
    subs, nc = list(c1["subs"]), list(c1["nc"])
    left_out = np.asarray(subs[0][:nc[0]])
    if not cover:
        subs, nc = subs[1:], nc[1:]    # the first subgraph's core vertices are in no core
    parts = import_parts(ctx, N, subs, nc)
    X, rep = gbe.sp2_submatrices(ctx, device_csr(H), parts, gbe.sp2_params(N // 2, prec=gbe.PREC_FP64, seq=c1["seq"]))
    n, width = gbe.assemble_width(ctx, X, parts)
    outs = []
    for kind in ("device", "pinned", "pageable"):
        if kind == "device":
            col = torch.full((n, width), 7, dtype=torch.int32, device="cuda")
            val = torch.full((n, width), float("nan"), dtype=torch.float64, device="cuda")
        elif kind == "pinned":
            col = torch.full((n, width), 7, dtype=torch.int32).pin_memory()
            val = torch.full((n, width), float("nan"), dtype=torch.float64).pin_memory()
        else:
            col = np.full((n, width), 7, dtype=np.int32)
            val = np.full((n, width), np.nan)
        gbe.assemble_D(ctx, X, parts, col, val)
        torch.cuda.synchronize()
        c = col.cpu().numpy() if torch.is_tensor(col) else col
        v = val.cpu().numpy() if torch.is_tensor(val) else val
        outs.append((c.copy(), v.copy()))
    for c, v in outs[1:]:
        np.testing.assert_array_equal(c, outs[0][0])
        np.testing.assert_array_equal(v, outs[0][1])
    c, v = outs[0]
    assert not np.isnan(v).any() and not (c == 7).all(axis=1).any()
    D = gbe.ell_to_dense(c, v, N)
    if cover:
        assert np.abs(D - c1["Dref"]).max() <= 1e-10
    else:
        assert np.all(c[left_out] == -1) and np.all(v[left_out] == 0.0)
        kept = np.setdiff1d(np.arange(N), left_out)
        assert np.abs(D[:, kept] - c1["Dref"][:, kept]).max() <= 1e-10
