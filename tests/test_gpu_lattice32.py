"""GPU parity at the benchmark's full size: the 32^3 lattice (N = 32,768), |H^2| >= 0.15 graph,
8^3 spatial cells (cores of 64 sites), SP2 launched as in the benchmark (CUDA graphs, default
launch configuration), checked on sampled subgraphs that the oracle computes one by one.

The oracle builds H from a k-d-tree neighbour search, the sampled halos from rows of H^2,
and applies the SP2 polynomial the GPU's FP64 run chose (its recorded branch sequence, global
Gershgorin bounds of the whole H) to each sampled submatrix.  Sampled: the smallest, the
largest and four random subgraphs.  Tolerances: FP64 1e-10, FP16X6 1e-6 (the mixed path's
bound); the assembled D rows of the sampled cores are checked against the same columns.
"""
import numpy as np
import pytest

import synth
from oracle import graph, hamiltonian, partition, sp2

pytestmark = pytest.mark.gpu

from tests.gpu_helpers import gbe, torch  # noqa: E402

L, THRESH, NCELL = 32, 0.15, (8, 8, 8)
TOL = {gbe.PREC_FP64: 1e-10, gbe.PREC_FP16X6: 1e-6, gbe.PREC_FP64TC: 1e-10}


@pytest.fixture(scope="module")
def ctx():
    return gbe.Context(0)


@pytest.fixture(scope="module")
def full(ctx):
    w = synth.lattice(L, seed=0)
    N = w["pos"].shape[0]
    st = gbe.sites(torch.from_numpy(w["pos"]).cuda(), torch.from_numpy(w["onsite"]).cuda(), w["box"])
    Hg = gbe.build_hamiltonian(ctx, st)
    G = gbe.build_graph(ctx, Hg.csr(), gbe.GRAPH_H2_THRESH, thresh=THRESH)
    parts = gbe.partition(ctx, G, gbe.PART_SPATIAL_CELLS, ncell=NCELL, site_struct=st)
    Ho = hamiltonian.build_h_tree(w["pos"], w["box"], w["onsite"])
    cores = partition.spatial_cores(w["pos"], w["box"], NCELL)
    cc, sub_ptr, sub_idx = parts.export()
    ms = np.diff(sub_ptr)
    rng = np.random.default_rng(1)
    picks = sorted(set([int(np.argmin(ms)), int(np.argmax(ms))] + list(rng.choice(len(cores), 4, replace=False))))
    # the FP64 run's own decisions (global FP64 traces, stall stop), as the benchmark runs it
    _, rep = gbe.sp2_submatrices(ctx, Hg.csr(), parts, gbe.sp2_params(N / 2.0, prec=gbe.PREC_FP64, n_max=48))
    return dict(w=w, N=N, st=st, Hg=Hg, parts=parts, Ho=Ho, cores=cores, cc=cc, sub_ptr=sub_ptr,
                sub_idx=sub_idx, picks=picks, ms=ms, seq=rep["seq"], stop=rep["stop"])


def test_full_size_partition_sampled(full):
    ms = full["ms"]
    assert len(full["cores"]) == len(full["cc"]) == 512
    assert 300 <= ms.min() and ms.max() <= 600, (ms.min(), ms.max())
    for s in full["picks"]:
        core = full["cores"][s]
        S = graph.h2_threshold_rows(full["Ho"], THRESH, core)
        (ref,), (nc,) = partition.subgraphs(S, [core])
        assert full["cc"][s] == nc
        np.testing.assert_array_equal(full["sub_idx"][full["sub_ptr"][s]:full["sub_ptr"][s + 1]], ref)


@pytest.mark.parametrize("prec", [gbe.PREC_FP64, gbe.PREC_FP16X6, gbe.PREC_FP64TC])
def test_full_size_sp2_sampled(ctx, full, prec):
    N, seq = full["N"], full["seq"]
    assert full["stop"] in ("stall", "tol") and len(seq) >= 10
    X, rep = gbe.sp2_submatrices(ctx, full["Hg"].csr(), full["parts"], gbe.sp2_params(N / 2.0, prec=prec, seq=seq))
    assert rep["iters"] == len(seq)
    eps = sp2.gershgorin(full["Ho"])
    assert abs(rep["eps"][0] - eps[0]) < 1e-12 and abs(rep["eps"][1] - eps[1]) < 1e-12
    n, width = gbe.assemble_width(ctx, X, full["parts"])
    col = torch.empty((n, width), dtype=torch.int32, device="cuda")
    val = torch.empty((n, width), dtype=torch.float64, device="cuda")
    gbe.assemble_D(ctx, X, full["parts"], col, val)
    torch.cuda.synchronize()
    worst = 0.0
    for s in full["picks"]:
        idx = full["sub_idx"][full["sub_ptr"][s]:full["sub_ptr"][s + 1]]
        c = int(full["cc"][s])
        _, _, (xs,) = sp2.sp2_graph(full["Ho"], [idx], [c], N // 2, seq=seq, eps=eps, return_subs=True)
        got = X.export(s, len(idx))
        worst = max(worst, float(np.abs(got - xs).max()))
        rows = torch.from_numpy(idx[:c].astype(np.int64)).cuda()
        ecol = col[rows].cpu().numpy()
        evals = val[rows].cpu().numpy()
        for j in range(c):
            keep = ecol[j] >= 0
            np.testing.assert_array_equal(np.sort(ecol[j][keep]), np.sort(idx))
            ref = dict(zip(idx, xs[:, j]))
            assert max(abs(v - ref[k]) for k, v in zip(ecol[j][keep], evals[j][keep])) <= TOL[prec]
    print(f"lattice 32^3, prec {prec}: {len(seq)} steps ({full['stop']}), max|dx| on sampled subgraphs {worst:.3e}")
    assert worst <= TOL[prec], worst
