"""GPU parity of the learned graph proposal: candidate pairs and features, the width-64
network's forward pass, its BCE gradient, Adam, the GBE_GRAPH_MLP graph, GPU training,
and what the trained network gains over the H^k-pattern graph.

Tolerances.  The kernels compute in FP32 with fp16-rounded weights (the 64 x 64 layer on
the tensor cores, its activations and back-propagated errors carried as fp16 hi + lo pairs,
relative error ~2^-21, with FP32 accumulation); the oracle in FP64 with the same rounded
weights.  A logit is a sum of products through three layers, so
its FP32 error is bounded by about (terms per dot product) x 2^-24 times the same
expression evaluated with absolute values (``abs_scale``); 1e-5 x abs_scale covers the
133-term depth with margin.  Features are FP32 roundings of FP64 values (log10f within
a few ulp).  Gradients are means over all pairs; they are compared per parameter block
against the block's largest entry.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import exact, graph, hamiltonian, mlp

pytestmark = pytest.mark.gpu

from tests.gpu_helpers import assembled_dense, device_array, gbe, torch  # noqa: E402

RCAND = 4.0


@pytest.fixture(scope="module")
def ctx():
    return gbe.Context(0)


def gpu_system(ctx, w):
    st = gbe.sites(torch.from_numpy(w["pos"]).cuda(), torch.from_numpy(w["onsite"]).cuda(), w["box"])
    Hg = gbe.build_hamiltonian(ctx, st)
    return st, Hg


def oracle_pairs(w, H, rows=None):
    I, J, R = mlp.candidate_pairs(w["pos"], w["box"], RCAND, rows=rows)
    return I, J, R, mlp.features(H, w["onsite"], I, J, R, RCAND)


def abs_scale(p, F):
    """|b3| + sum |w3| (|b2| + |W2| (|b1| + |W1| |f|)) with the fp16-rounded weights."""
    W1, b1, W2, b2, w3, b3 = mlp.unpack(mlp.fp16_round(p))
    a1 = np.abs(F) @ np.abs(W1).T + np.abs(b1)
    a2 = a1 @ np.abs(W2).T + np.abs(b2)
    return a2 @ np.abs(w3) + abs(b3)


def make_params(seed):
    """Initial parameters with non-zero biases, so that every term of the network is exercised."""
    rng = np.random.default_rng(seed)
    p = mlp.init_params(seed).astype(np.float64)
    W1, b1, W2, b2, w3, b3 = (slice(0, 320), slice(320, 384), slice(384, 4480), slice(4480, 4544),
                              slice(4544, 4608), slice(4608, 4609))
    for s in (b1, b2):
        p[s] = rng.normal(0.0, 0.3, s.stop - s.start)
    p[b3] = 0.2
    return p.astype(np.float32)


@pytest.fixture(scope="module")
def dis(ctx):
    w = synth.disordered(1500, seed=7)
    H = hamiltonian.build_h(w["pos"], w["box"], w["onsite"])
    st, Hg = gpu_system(ctx, w)
    P = gbe.pairs_build(ctx, st, Hg.csr(), RCAND)
    I, J, R, F = oracle_pairs(w, H)
    return dict(w=w, H=H, st=st, Hg=Hg, P=P, I=I, J=J, R=R, F=F)


@pytest.mark.parametrize("kind", ["lattice", "disordered", "dense"])
def test_pairs_and_features(ctx, kind, dis):
    """Pairs, their order and features against the oracle.  "lattice" and "disordered" take the
    single-pass search (candidates staged per site) and the candidate-keyed (H^2)_ij table;
    "dense", density 3/a^3 (~800 candidates within 4a), has sites with more candidates than a
    staging slot (512), so the build runs the filling pass, and more than half the table, so
    those sites take the ordered row merge for (H^2)_ij."""
    if kind == "disordered":
        w, H, P, I, J, F = dis["w"], dis["H"], dis["P"], dis["I"], dis["J"], dis["F"]
    else:
        w = synth.lattice(10, seed=5) if kind == "lattice" else synth.disordered(2000, density=3.0, seed=8)
        H = hamiltonian.build_h(w["pos"], w["box"], w["onsite"])
        st, Hg = gpu_system(ctx, w)
        P = gbe.pairs_build(ctx, st, Hg.csr(), RCAND)
        I, J, _, F = oracle_pairs(w, H)
    rp, jg, fg = P.export()
    N = len(w["pos"])
    assert P.info() == (N, len(I))
    np.testing.assert_array_equal(rp, np.concatenate([[0], np.cumsum(np.bincount(I, minlength=N))]))
    np.testing.assert_array_equal(jg, J)
    np.testing.assert_allclose(fg[:, 0], F[:, 0], rtol=0, atol=2e-7)
    np.testing.assert_allclose(fg[:, 1], F[:, 1], rtol=0, atol=2e-7)
    np.testing.assert_allclose(fg[:, 2:], F[:, 2:], rtol=1.2e-7, atol=0)
    # every feature is symmetric in (i, j) bit for bit
    key = I.astype(np.int64) * N + J
    back = np.searchsorted(key, J.astype(np.int64) * N + I)
    np.testing.assert_array_equal(fg, fg[back])


def test_forward_matches_oracle(ctx, dis):
    p = make_params(3)
    M = gbe.mlp_create(ctx)
    M.set_params(p)
    np.testing.assert_array_equal(M.get_params(), p)
    npairs = dis["P"].info()[1]
    z = torch.empty(npairs, dtype=torch.float32, device="cuda")
    M.forward(dis["P"], z)
    torch.cuda.synchronize()
    zg = z.cpu().numpy().astype(np.float64)
    zo = mlp.forward(p, dis["F"])
    err = np.abs(zg - zo) / abs_scale(p, dis["F"])
    assert err.max() <= 1e-5, err.max()
    # the logits are symmetric in (i, j) bit for bit: the features are
    key = dis["I"].astype(np.int64) * 1500 + dis["J"]
    back = np.searchsorted(key, dis["J"].astype(np.int64) * 1500 + dis["I"])
    np.testing.assert_array_equal(zg, zg[back])


def block_slices():
    return dict(W1=slice(0, 320), b1=slice(320, 384), W2=slice(384, 4480), b2=slice(4480, 4544),
                w3=slice(4544, 4608), b3=slice(4608, 4609))


@pytest.mark.parametrize("tau", [1e-2, 1e-5])
def test_gradient_matches_oracle(ctx, dis, tau):
    D, _ = exact.density_matrix(dis["H"], 750)
    y = mlp.labels(D, dis["I"], dis["J"], tau)
    labels = torch.from_numpy(y.astype(np.uint8)).cuda()
    p = make_params(4)
    M = gbe.mlp_create(ctx)
    M.set_params(p)
    loss_g, g_g = M.gradient(dis["P"], labels)
    loss_o, g_o = mlp.loss_and_grad(p, dis["F"], y)
    assert abs(loss_g - loss_o) <= 1e-6 * loss_o
    for name, s in block_slices().items():
        ref = np.abs(g_o[s]).max()
        assert np.abs(g_g[s] - g_o[s]).max() <= 2e-4 * ref + 1e-9, name
    # the reduction order is fixed: a second call gives the same bits
    loss_2, g_2 = M.gradient(dis["P"], labels)
    assert loss_2 == loss_g
    np.testing.assert_array_equal(g_2, g_g)


def test_adam_first_step_and_trajectory(ctx, dis):
    D, _ = exact.density_matrix(dis["H"], 750)
    y = mlp.labels(D, dis["I"], dis["J"], 1e-2)
    labels = torch.from_numpy(y.astype(np.uint8)).cuda()
    p0 = make_params(5)
    lr = 1e-3
    M = gbe.mlp_create(ctx)
    M.set_params(p0)
    M.gradient(dis["P"], labels)
    M.adam_step(lr)
    p1 = M.get_params().astype(np.float64)
    _, g_o = mlp.loss_and_grad(p0, dis["F"], y)
    d = p1 - p0.astype(np.float64)
    # first bias-corrected step: -lr g / (|g| + eps), i.e. -lr sign(g) where g is well above
    # the FP32 gradient error; exactly zero where the gradient is exactly zero (dead units)
    big = np.abs(g_o) > 1e-3 * np.abs(g_o).max()
    ulp = np.spacing(np.abs(p0).astype(np.float32)).astype(np.float64)
    np.testing.assert_array_less(np.abs(d[big] + lr * g_o[big] / (np.abs(g_o[big]) + 1e-8)), 1e-6 * lr + ulp[big])
    assert np.all(d[g_o == 0.0] == 0.0)
    # 40 steps: the loss follows the oracle's Adam trajectory
    M.set_params(p0)
    steps = 40
    loss_g = M.train(dis["P"], labels, steps, lr)
    p, m, v = p0.astype(np.float64), np.zeros(p0.size), np.zeros(p0.size)
    for t in range(1, steps + 1):
        loss_o, g = mlp.loss_and_grad(p, dis["F"], y)
        p, m, v = mlp.adam_step(p, g, m, v, t, lr)
    assert abs(loss_g - loss_o) <= 1e-3 * loss_o, (loss_g, loss_o)


def test_mlp_graph_matches_oracle(ctx, dis):
    p = make_params(6)
    zo = mlp.forward(p, dis["F"])
    cut = float(np.quantile(zo, 0.7))
    M = gbe.mlp_create(ctx)
    M.set_params(p)
    G = gbe.build_graph(ctx, dis["Hg"].csr(), gbe.GRAPH_MLP, site_struct=dis["st"], mlp=M, rcand=RCAND,
                        logit_cut=cut)
    rp, col = G.export()
    N = 1500
    Gg = sp.csr_matrix((np.ones(len(col), dtype=bool), col, rp), shape=(N, N))
    Go = mlp.graph_from_logits(dis["H"], dis["I"], dis["J"], zo, cut)
    diff = (Gg != Go).tocoo()
    # pairs may differ only where the oracle logit lies within the FP32 error bound of the cut
    margin = 1e-5 * abs_scale(p, dis["F"])
    near = {(i, j) for i, j, z, e in zip(dis["I"], dis["J"], zo, margin) if abs(z - cut) <= e}
    assert all((i, j) in near or (j, i) in near for i, j in zip(diff.row, diff.col))
    assert Go.nnz > (dis["H"] != 0).nnz   # the network adds edges beyond the pattern of H
    assert np.all(np.diff(rp) > 0)


# ------------------------------------------------------------------ training and its gain
def lattice_labels(L, seed, tau):
    w = synth.lattice(L, seed=seed)
    H = hamiltonian.build_h(w["pos"], w["box"], w["onsite"])
    D, _ = exact.density_matrix(H, H.shape[0] // 2)
    return w, H, D


def graph_sp2_error(ctx, Hg, G, st, N, D_exact, ncell, prec=gbe.PREC_FP64):
    parts = gbe.partition(ctx, G, gbe.PART_SPATIAL_CELLS, ncell=ncell, site_struct=st)
    cc, sub_ptr, _ = parts.export()
    m = np.diff(sub_ptr).astype(np.float64)
    X, rep = gbe.sp2_submatrices(ctx, Hg.csr(), parts, gbe.sp2_params(N // 2, prec=prec))
    Dg, _, _ = assembled_dense(ctx, X, parts, N)
    return dict(err=float(np.abs(Dg - D_exact).max()), mean_m=float(m.mean()), flops=float(np.sum(m ** 3)),
                edges=G.size()[1] / N, iters=rep["iters"])


@pytest.mark.parametrize("tau", [1e-2, 1e-5])
def test_labels_from_assembled_D(ctx, dis, tau):
    """gbe_mlp_labels against the oracle's labels of the same D: the GPU's graph SP2 D of the
    1500-site disordered system (|H^2| >= 0.1 graph, cores from 3^3 cells), copied to the
    host.  Pairs outside a core's subgraph have no entry in D and get label 0.  Bit for bit."""
    N, st, Hg, P, I, J = 1500, dis["st"], dis["Hg"], dis["P"], dis["I"], dis["J"]
    G = gbe.build_graph(ctx, Hg.csr(), gbe.GRAPH_H2_THRESH, thresh=0.1)
    parts = gbe.partition(ctx, G, gbe.PART_SPATIAL_CELLS, ncell=(3, 3, 3), site_struct=st)
    X, _ = gbe.sp2_submatrices(ctx, Hg.csr(), parts, gbe.sp2_params(N // 2, prec=gbe.PREC_FP64))
    n, width = gbe.assemble_width(ctx, X, parts)
    col = torch.empty((n, width), dtype=torch.int32, device="cuda")
    val = torch.empty((n, width), dtype=torch.float64, device="cuda")
    gbe.assemble_D(ctx, X, parts, col, val)
    lab = torch.full((len(I),), 7, dtype=torch.uint8, device="cuda")
    gbe.mlp_labels(ctx, P, col, val, tau, lab)
    torch.cuda.synchronize()
    D = gbe.ell_to_dense(col.cpu().numpy(), val.cpu().numpy(), N)
    y = mlp.labels(D, I, J, tau).astype(np.uint8)
    assert np.array_equal(lab.cpu().numpy(), y)
    absent = D[I, J] == 0.0
    assert absent.any() and 0.0 < y.mean() < 1.0
    with pytest.raises(gbe.GbeError):
        gbe.mlp_labels(ctx, P, col.cpu(), val.cpu(), tau, lab)
    # labels in host memory are refused before the kernel could write them
    with pytest.raises(gbe.GbeError) as e:
        gbe.mlp_labels(ctx, P, col, val, tau, np.zeros(len(I), np.uint8))
    assert e.value.code == gbe.GBE_EINVAL and "device memory" in str(e.value)


TRAIN_SEEDS = range(1000, 1008)   # eight seeded, jittered 16^3 lattices (4096 sites each)


def test_training_and_gain_over_hk(ctx, capsys):
    """Train on eight seeded, jittered 16^3 lattices (labels |D_ij| >= 1e-2 from exact
    diagonalisation; one Adam step per system in turn, 40 passes), then build graphs for an
    unseen 16^3 lattice and run FP64-grade graph SP2 (FP64TC) on each with cores of 8
    sites: the network's graph reaches an error the H^1 graph does not, at a fraction of
    the cost of the smallest H^k graph (k = 2) that reaches it, and prunes the candidate
    ball."""
    tau = 1e-2
    sets = []
    for seed in TRAIN_SEEDS:
        w, H, D = lattice_labels(16, seed, tau)
        st, Hg = gpu_system(ctx, w)
        P = gbe.pairs_build(ctx, st, Hg.csr(), RCAND)
        I, J, _ = mlp.candidate_pairs(w["pos"], w["box"], RCAND)
        y = mlp.labels(D, I, J, tau)
        sets.append((P, torch.from_numpy(y.astype(np.uint8)).cuda(), st, Hg, float(y.mean())))
    M = gbe.mlp_create(ctx)
    M.set_params(mlp.init_params(0))
    loss0 = float(np.mean([M.gradient(P, lab)[0] for P, lab, *_ in sets]))
    for _ in range(40):
        for P, lab, *_ in sets:
            M.train(P, lab, 1, 3e-3)
    loss = float(np.mean([M.gradient(P, lab)[0] for P, lab, *_ in sets]))
    assert loss < 0.75 * loss0 and loss < 0.3, (loss0, loss)

    wt, Ht, Dt = lattice_labels(16, 1199, tau)
    N = Ht.shape[0]
    stt, Hgt = gpu_system(ctx, wt)
    # accuracy on the unseen system, from the network's own logits
    Pt = gbe.pairs_build(ctx, stt, Hgt.csr(), RCAND)
    It, Jt, _ = mlp.candidate_pairs(wt["pos"], wt["box"], RCAND)
    yt = mlp.labels(Dt, It, Jt, tau)
    z = torch.empty(len(It), dtype=torch.float32, device="cuda")
    M.forward(Pt, z)
    acc = float(np.mean((z.cpu().numpy() >= 0) == (yt > 0.5)))
    assert acc > 0.85, acc

    ncell = (8, 8, 8)
    res = {}
    for k in (1, 2):
        res[f"H^{k}"] = graph_sp2_error(ctx, Hgt, gbe.build_graph(ctx, Hgt.csr(), gbe.GRAPH_HK_PATTERN, k=k), stt, N,
                                        Dt, ncell, gbe.PREC_FP64TC)
    for cut in (-6.0, -2.0):
        G = gbe.build_graph(ctx, Hgt.csr(), gbe.GRAPH_MLP, site_struct=stt, mlp=M, rcand=RCAND, logit_cut=cut)
        res[f"MLP cut {cut:g}"] = graph_sp2_error(ctx, Hgt, G, stt, N, Dt, ncell, gbe.PREC_FP64TC)
    G = gbe.build_graph(ctx, Hgt.csr(), gbe.GRAPH_MLP, site_struct=stt, mlp=M, rcand=RCAND, logit_cut=-1e30)
    res["ball r<4"] = graph_sp2_error(ctx, Hgt, G, stt, N, Dt, ncell, gbe.PREC_FP64TC)
    with capsys.disabled():
        print(f"\ntrained on {len(sets)} 16^3 lattices (positive rate {np.mean([s[4] for s in sets]):.3f}): "
              f"loss {loss0:.4f} -> {loss:.4f}, unseen 16^3 accuracy {acc:.4f}")
        for name, r in res.items():
            print(f"  {name:12s} edges/row {r['edges']:7.1f}  mean m {r['mean_m']:7.1f}  "
                  f"sum m^3 {r['flops']:.3e}  max|D-D_exact| {r['err']:.3e}")
    mlp6, h1, h2 = res["MLP cut -6"], res["H^1"], res["H^2"]
    assert mlp6["err"] < h1["err"]                 # H^1 does not reach the network graph's error ...
    assert h2["err"] <= mlp6["err"]                # ... H^2 is the smallest H^k graph that does
    assert mlp6["flops"] * 3 < h2["flops"]         # ... at three or more times the network graph's cost
    assert mlp6["flops"] < res["ball r<4"]["flops"]  # the network prunes the candidate ball


def test_full_size_inference_sampled(ctx):
    """1,048,576-site disordered system (box 101.6 a): candidate pairs, features and logits of
    the whole system on the GPU, sampled rows against the oracle computed row by row."""
    N = 1 << 20
    w = synth.disordered(N, seed=2024)
    st, Hg = gpu_system(ctx, w)
    P = gbe.pairs_build(ctx, st, Hg.csr(), RCAND)
    n, npairs = P.info()
    assert n == N and 250 * N < npairs < 290 * N
    p = make_params(8)
    M = gbe.mlp_create(ctx)
    M.set_params(p)
    z = torch.empty(npairs, dtype=torch.float32, device="cuda")
    M.forward(P, z)
    rp_d, j_d, f_d = P.device()
    rp = device_array(rp_d, N + 1, "<i8")
    rows = np.sort(np.random.default_rng(1).choice(N, 6, replace=False))
    I, J, R = mlp.candidate_pairs(w["pos"], w["box"], RCAND, rows=rows)
    touched = np.union1d(rows, J)
    Hrows = hamiltonian.build_h(w["pos"], w["box"], w["onsite"], rows=touched, chunk=8)
    # N x N matrix holding only the touched rows (the features need rows i and j only)
    Hr = (sp.csr_matrix((np.ones(len(touched)), (touched, np.arange(len(touched)))), shape=(N, len(touched)))
          @ Hrows).tocsr()
    F = mlp.features(Hr, w["onsite"], I, J, R, RCAND)
    zo = mlp.forward(p, F)
    scale = abs_scale(p, F)
    o = 0
    zall = z.cpu().numpy()
    for i in rows:
        cnt = int(np.sum(I == i))
        a, b = int(rp[i]), int(rp[i + 1])
        assert b - a == cnt
        jg = device_array(j_d + 4 * a, cnt, "<i4")
        fg = device_array(f_d + 20 * a, 5 * cnt, "<f4").reshape(cnt, 5)
        np.testing.assert_array_equal(jg, J[o:o + cnt])
        np.testing.assert_allclose(fg[:, :2], F[o:o + cnt, :2], rtol=0, atol=2e-7)
        np.testing.assert_allclose(fg[:, 2:], F[o:o + cnt, 2:], rtol=1.2e-7, atol=0)
        assert np.all(np.abs(zall[a:b] - zo[o:o + cnt]) <= 1e-5 * scale[o:o + cnt])
        o += cnt
