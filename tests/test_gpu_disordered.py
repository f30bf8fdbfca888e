"""GPU parity on the disordered liquid-like model: uneven halos, every precision.

Uniform random sites at density 1/a^3, onsite N(+-1, 0.1) by species, the lattice's
hopping; cores of ~64 sites from spatial cells of ~4a; graph |H^2| >= 0.1, which spreads
the submatrix sizes over several 128-wide buckets.

(a) A 4096-site sample (box 16a, 4x4x4 cells): the whole GPU chain (H, graph, partition,
    SP2, assembly) against the oracle's chain; the oracle's free-running branch sequence
    is replayed on the GPU.
(b) The full 131,072-site system (box 50.8a, 13x13x13 cells): the GPU chain at full size,
    checked on sampled submatrices that the oracle computes one by one (its H from a
    k-d-tree neighbour search, the sampled halos from rows of H^2, and the SP2 polynomial
    of (a)'s branch sequence applied to each sampled submatrix).
Tolerances: FP64 1e-10.  FP64TC (the FP64-grade tensor-core squaring) 1e-10 on the full-size
sampled subgraphs and 5e-10 on the 4096-site sample, whose amplification is the largest:
one FP32 rounding per MMA into its fourth accumulator (|value| ~ 4 in units of 2^-30, so
~2^-52 of an element per addition, 9 products x K/16 additions) and the dropped 2^-50
level leave a squaring within a few 1e-15, about ten times the FP64 DFMA path's own
rounding, and the same amplification turns that into ~1.5e-10.  This model is near-metallic (HOMO-LUMO gap ~0.02 eV against a
Gershgorin range of ~50 eV; 56 SP2 steps before the idempotency error stalls), and an SP2
expansion amplifies a perturbation of an early iterate near the chemical potential by the
slope of the remaining polynomial: the FP64 path's own rounding (~1e-16) reaches ~1e-12 in D.
The FP16X6 split represents every element to ~2^-34, which the same amplification turns into
~2e-6 (a CPU emulation of the split with exact accumulation gives 1.7e-6 on the 4096-site
sample), so FP16X6 and BF16X3 miss the mixed path's 1e-6 bound on this model: they are held
here to what they reach, 1e-5 (FP16X6) and 5e-2 (BF16X3, ~2^-17 per element), and meet 1e-6
on the gapped lattice only.  The mixed path that meets 1e-6 on this model is FP64TC, held
to the FP64 bounds above.
"""
import numpy as np
import pytest

import synth
from oracle import graph, hamiltonian, partition, sp2

pytestmark = pytest.mark.gpu

from tests.gpu_helpers import assembled_dense, gbe, torch  # noqa: E402

THRESH = 0.1
TOL = {0: 1e-10, 1: 1e-5, 2: 5e-2, 3: 1e-10}
TOL_SAMPLE = {**TOL, 3: 5e-10}


@pytest.fixture(scope="module")
def ctx():
    return gbe.Context(0)


def gpu_chain(ctx, w, ncell):
    st = gbe.sites(torch.from_numpy(w["pos"]).cuda(), torch.from_numpy(w["onsite"]).cuda(), w["box"])
    Hg = gbe.build_hamiltonian(ctx, st)
    G = gbe.build_graph(ctx, Hg.csr(), gbe.GRAPH_H2_THRESH, thresh=THRESH)
    parts = gbe.partition(ctx, G, gbe.PART_SPATIAL_CELLS, ncell=ncell, site_struct=st)
    return st, Hg, parts


@pytest.fixture(scope="module")
def sample():
    w = synth.disordered(4096, seed=0)
    H = hamiltonian.build_h(w["pos"], w["box"], w["onsite"])
    S = graph.h2_threshold(H, THRESH)
    subs, nc = partition.subgraphs(S, partition.spatial_cores(w["pos"], w["box"], (4, 4, 4)))
    D, log = sp2.sp2_graph(H, subs, nc, 2048, n_max=60)
    return dict(w=w, H=H, subs=subs, nc=nc, D=D.toarray(), seq=log.seq, stop=log.stop)


def test_sample_partition_is_uneven_and_exact(ctx, sample):
    _, _, parts = gpu_chain(ctx, sample["w"], (4, 4, 4))
    cc, sub_ptr, sub_idx = parts.export()
    assert list(cc) == list(sample["nc"])
    subs_g = np.split(sub_idx, sub_ptr[1:-1])
    assert all(np.array_equal(a, b) for a, b in zip(subs_g, sample["subs"]))
    ms = np.array([len(s) for s in sample["subs"]])
    # several 128-wide buckets
    assert len(np.unique((ms + 127) // 128)) >= 2, (ms.min(), ms.max())


@pytest.mark.parametrize("prec", [gbe.PREC_FP64, gbe.PREC_FP16X6, gbe.PREC_BF16X3, gbe.PREC_FP64TC])
def test_sample_chain_parity(ctx, sample, prec):
    st, Hg, parts = gpu_chain(ctx, sample["w"], (4, 4, 4))
    X, rep = gbe.sp2_submatrices(ctx, Hg.csr(), parts, gbe.sp2_params(2048, prec=prec, seq=sample["seq"]))
    assert rep["iters"] == len(sample["seq"])
    D, _, _ = assembled_dense(ctx, X, parts, 4096)
    err = np.abs(D - sample["D"]).max()
    print(f"disordered 4096, prec {prec}: {len(sample['seq'])} steps ({sample['stop']}), max|dD| {err:.3e}")
    assert err <= TOL_SAMPLE[prec], err


def test_sample_free_running_decisions(ctx, sample):
    st, Hg, parts = gpu_chain(ctx, sample["w"], (4, 4, 4))
    _, rep = gbe.sp2_submatrices(ctx, Hg.csr(), parts, gbe.sp2_params(2048, prec=gbe.PREC_FP64, n_max=60))
    assert rep["stop"] == sample["stop"]
    assert rep["seq"] == sample["seq"]


@pytest.fixture(scope="module")
def full(ctx, sample):
    N = 131072
    w = synth.disordered(N, seed=0)
    ncell = (13, 13, 13)
    st, Hg, parts = gpu_chain(ctx, w, ncell)
    Ho = hamiltonian.build_h_tree(w["pos"], w["box"], w["onsite"])
    cores = partition.spatial_cores(w["pos"], w["box"], ncell)
    cc, sub_ptr, sub_idx = parts.export()
    rng = np.random.default_rng(0)
    ms = np.diff(sub_ptr)
    # sampled subgraphs: the smallest, the largest and four random ones
    picks = sorted(set([int(np.argmin(ms)), int(np.argmax(ms))] + list(rng.choice(len(cores), 4, replace=False))))
    return dict(w=w, N=N, st=st, Hg=Hg, parts=parts, Ho=Ho, cores=cores, cc=cc, sub_ptr=sub_ptr,
                sub_idx=sub_idx, picks=picks, ms=ms)


def test_full_size_partition_sampled(full):
    assert len(full["cores"]) == len(full["cc"])
    ms = full["ms"]
    print(f"disordered 131072: {len(ms)} subgraphs, m_s {ms.min()}..{ms.max()} (median {np.median(ms):.0f})")
    for s in full["picks"]:
        core = full["cores"][s]
        S = graph.h2_threshold_rows(full["Ho"], THRESH, core)
        (ref,), (nc,) = partition.subgraphs(S, [core])
        assert full["cc"][s] == nc
        np.testing.assert_array_equal(full["sub_idx"][full["sub_ptr"][s]:full["sub_ptr"][s + 1]], ref)


@pytest.mark.parametrize("prec", [gbe.PREC_FP64, gbe.PREC_FP16X6, gbe.PREC_BF16X3, gbe.PREC_FP64TC])
def test_full_size_sp2_sampled(ctx, full, sample, prec):
    N = full["N"]
    seq = sample["seq"]
    X, rep = gbe.sp2_submatrices(ctx, full["Hg"].csr(), full["parts"], gbe.sp2_params(N // 2, prec=prec, seq=seq))
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
        # the oracle applies the same polynomial (global bounds, the given sequence) to this submatrix
        _, _, (xs,) = sp2.sp2_graph(full["Ho"], [idx], [c], N // 2, seq=seq, eps=eps, return_subs=True)
        got = X.export(s, len(idx))
        worst = max(worst, float(np.abs(got - xs).max()))
        # assembled D: ELL row of core site idx[j] holds column idx[j] of D
        rows = torch.from_numpy(idx[:c].astype(np.int64)).cuda()
        ecol = col[rows].cpu().numpy()
        evals = val[rows].cpu().numpy()
        for j in range(c):
            m = ecol[j] >= 0
            order = np.argsort(ecol[j][m])
            np.testing.assert_array_equal(ecol[j][m][order], np.sort(idx))
            ref = dict(zip(idx, xs[:, j]))
            assert max(abs(v - ref[k]) for k, v in zip(ecol[j][m], evals[j][m])) <= TOL[prec]
    print(f"disordered 131072, prec {prec}: max|dx| on sampled subgraphs {worst:.3e}")
    assert worst <= TOL[prec], worst
