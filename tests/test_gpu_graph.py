"""GPU parity of H build, graph builders (Eq. 2, Eq. 8, H^k) and partitions against the oracle.

Integer structures (graph patterns, core lists, halo lists) must match exactly; H values
to 1e-14 relative (CUDA exp vs NumPy exp), pairs within 1e-12 of the cutoff excepted.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import graph, hamiltonian, partition, sp2

pytestmark = pytest.mark.gpu

from tests.gpu_helpers import assembled_dense, device_array, device_csr, gbe, host_csr, torch  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    return gbe.Context(0)


def h_to_scipy(Hg):
    """Host copy of a library-owned device CSR (read through __cuda_array_interface__)."""
    v = Hg.csr()
    n, nnz = v.n, v.nnz
    rp = device_array(v.rowptr, n + 1, "<i8")
    ci = device_array(v.col, nnz, "<i4")
    va = device_array(v.val, nnz, "<f8")
    return sp.csr_matrix((va, ci, rp), shape=(n, n))


def compare_h(Hg, Ho, pos, box, rcut=2.5):
    Hg = Hg.tocsr(); Ho = Ho.tocsr()
    assert Hg.shape == Ho.shape
    dg = Hg.toarray() if Hg.shape[0] <= 4096 else None
    do = Ho.toarray() if Ho.shape[0] <= 4096 else None
    pg = dg != 0
    po = do != 0
    diff = np.argwhere(pg != po)
    for i, j in diff:   # only pairs sitting on the cutoff may differ
        d = pos[i] - pos[j]
        d -= box * np.round(d / box)
        assert abs(np.sqrt((d * d).sum()) - rcut) < 1e-12
    both = pg & po
    np.testing.assert_allclose(dg[both], do[both], rtol=1e-14, atol=0)


@pytest.mark.parametrize("kind", ["lattice", "disordered", "dense"])
def test_hamiltonian_parity(ctx, kind):
    """"dense": density 3/a^3, ~196 neighbours per row, longer than the single-pass build's
    128-entry staging rows, so the build takes its second neighbour search."""
    if kind == "lattice":
        w = synth.lattice(8, seed=2)
    elif kind == "disordered":
        w = synth.disordered(1500, seed=7)
    else:
        w = synth.disordered(2000, density=3.0, seed=8)
    st = gbe.sites(torch.from_numpy(w["pos"]).cuda(), torch.from_numpy(w["onsite"]).cuda(), w["box"])
    Hg = h_to_scipy(gbe.build_hamiltonian(ctx, st))
    Ho = hamiltonian.build_h(w["pos"], w["box"], w["onsite"])
    compare_h(Hg, Ho, w["pos"], w["box"])
    rowlen = np.diff(Hg.indptr)
    assert (rowlen.max() > 128) == (kind == "dense"), rowlen.max()
    # rows sorted, diagonal present
    assert all(np.all(np.diff(Hg.indices[Hg.indptr[i]:Hg.indptr[i + 1]]) > 0) for i in range(0, Hg.shape[0], 97))
    np.testing.assert_array_equal(Hg.diagonal(), w["onsite"])


def test_hamiltonian_host_sites(ctx):
    w = synth.lattice(6, seed=9)
    st = gbe.sites(w["pos"], w["onsite"], w["box"])
    Hg = h_to_scipy(gbe.build_hamiltonian(ctx, st))
    compare_h(Hg, hamiltonian.build_h(w["pos"], w["box"], w["onsite"]), w["pos"], w["box"])


def export_graph(G, n):
    rp, ci = G.export()
    return sp.csr_matrix((np.ones(len(ci), dtype=bool), ci, rp), shape=(n, n))


def assert_same_pattern(A, B):
    A = sp.csr_matrix(A, dtype=bool); B = sp.csr_matrix(B, dtype=bool)
    A.sort_indices(); B.sort_indices()
    np.testing.assert_array_equal(A.indptr, B.indptr)
    np.testing.assert_array_equal(A.indices, B.indices)


@pytest.fixture(scope="module")
def lat():
    w = synth.lattice(8, seed=0)
    H = hamiltonian.build_h(w["pos"], w["box"], w["onsite"])
    return w, H


@pytest.mark.parametrize("thr", [1e-5, 1e-2, 0.3])
def test_graph_h2_threshold(ctx, lat, thr):
    w, H = lat
    G = gbe.build_graph(ctx, device_csr(H), gbe.GRAPH_H2_THRESH, thresh=thr)
    assert_same_pattern(export_graph(G, H.shape[0]), graph.h2_threshold(H, thr))


@pytest.mark.parametrize("k", [1, 2, 3])
def test_graph_hk_pattern(ctx, lat, k):
    w, H = lat
    G = gbe.build_graph(ctx, host_csr(H), gbe.GRAPH_HK_PATTERN, k=k)
    assert_same_pattern(export_graph(G, H.shape[0]), graph.hk_pattern(H, k))


def synthetic_ell(N, W, seed):
    """Random ELL 'density matrix' (row i = column i of D) with uneven row lengths."""
    rng = np.random.default_rng(seed)
    col = -np.ones((N, W), dtype=np.int32)
    val = np.zeros((N, W))
    for i in range(N):
        k = rng.integers(1, W + 1)
        cols = np.sort(rng.choice(N, size=k, replace=False))
        col[i, :k] = cols
        val[i, :k] = rng.normal(size=k) * 10.0 ** rng.uniform(-7, 0, size=k)
    return col, val


def ell_to_scipy_D(col, val, N):
    rows, cols, vals = [], [], []
    for i in range(N):
        m = col[i] >= 0
        rows.append(col[i][m]); cols.append(np.full(m.sum(), i)); vals.append(val[i][m])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))


@pytest.mark.parametrize("mode", ["d", "eq8"])
def test_graph_from_prior_d(ctx, lat, mode):
    w, H = lat
    N = H.shape[0]
    col, val = synthetic_ell(N, 40, seed=1)
    Do = ell_to_scipy_D(col, val, N)
    tau = 1e-4
    ell = gbe.ell_struct(torch.from_numpy(col).cuda(), torch.from_numpy(val).cuda())
    if mode == "d":
        G = gbe.build_graph(ctx, device_csr(H), gbe.GRAPH_D_THRESH, thresh=tau, D_prev=ell)
        ref = graph.d_threshold(Do, tau)
    else:
        G = gbe.build_graph(ctx, device_csr(H), gbe.GRAPH_EQ8_SYMBOLIC, thresh=tau, D_prev=ell)
        ref = graph.eq8_symbolic(Do, H, tau)
    assert_same_pattern(export_graph(G, N), ref)


def export_parts(P):
    cc, sp_, si = P.export()
    return [si[sp_[s]:sp_[s + 1]] for s in range(len(cc))], cc


@pytest.mark.parametrize("ncell", [(4, 4, 4), (3, 5, 2)])
def test_partition_spatial_cells(ctx, lat, ncell):
    w, H = lat
    N = H.shape[0]
    S = graph.h2_threshold(H, 1e-3)
    G = gbe.build_graph(ctx, device_csr(H), gbe.GRAPH_H2_THRESH, thresh=1e-3)
    st = gbe.sites(torch.from_numpy(w["pos"]).cuda(), torch.from_numpy(w["onsite"]).cuda(), w["box"])
    Pg = gbe.partition(ctx, G, gbe.PART_SPATIAL_CELLS, ncell=ncell, site_struct=st)
    subs_g, nc_g = export_parts(Pg)
    subs_o, nc_o = partition.subgraphs(S, partition.spatial_cores(w["pos"], w["box"], ncell))
    np.testing.assert_array_equal(nc_g, nc_o)
    assert len(subs_g) == len(subs_o)
    for a, b in zip(subs_g, subs_o):
        np.testing.assert_array_equal(a, b)


def test_partition_index_blocks_two_hops(ctx, lat):
    w, H = lat
    N = H.shape[0]
    G = gbe.build_graph(ctx, device_csr(H), gbe.GRAPH_HK_PATTERN, k=2)
    Pg = gbe.partition(ctx, G, gbe.PART_INDEX_BLOCKS, core_size=37)
    subs_g, nc_g = export_parts(Pg)
    subs_o, nc_o = partition.subgraphs(graph.hk_pattern(H, 2), partition.block_cores(N, 37))
    np.testing.assert_array_equal(nc_g, nc_o)
    for a, b in zip(subs_g, subs_o):
        np.testing.assert_array_equal(a, b)


def test_partition_capacity_error(ctx, lat):
    w, H = lat
    G = gbe.build_graph(ctx, device_csr(H), gbe.GRAPH_HK_PATTERN, k=2)
    with pytest.raises(gbe.GbeError) as e:
        gbe.partition(ctx, G, gbe.PART_INDEX_BLOCKS, core_size=8, max_sub=64)
    assert e.value.code == gbe.GBE_ECAPACITY


@pytest.mark.parametrize("prec", [gbe.PREC_FP16X6, gbe.PREC_FP64])
def test_partition_autotune_picks_cheapest(ctx, prec):
    """Cost-driven partition size on the 21^3 lattice (|H^2| >= 0.15 graph): every candidate
    cell grid is partitioned and costed by the modelled squaring time of one SP2 step
    (checked here against the formula on the exported subgraph sizes); a grid whose
    subgraphs exceed what the gather holds (one cell: 9261 sites, above 8192) is infeasible;
    the cheapest one is returned."""
    w = synth.lattice(21, seed=3)
    st = gbe.sites(torch.from_numpy(w["pos"]).cuda(), torch.from_numpy(w["onsite"]).cuda(), w["box"])
    Hg = gbe.build_hamiltonian(ctx, st)
    G = gbe.build_graph(ctx, Hg.csr(), gbe.GRAPH_H2_THRESH, thresh=0.15)
    cands = [(1, 1, 1), (3, 3, 3), (7, 7, 7), (21, 21, 21)]
    parts, best, cost = gbe.partition_autotune(ctx, G, cands, prec=prec, site_struct=st)
    assert np.isinf(cost[0]) and np.all(np.isfinite(cost[1:]))
    for i, c in enumerate(cands[1:], start=1):
        _, sp, _ = gbe.partition(ctx, G, gbe.PART_SPATIAL_CELLS, ncell=c, site_struct=st).export()
        m = np.diff(sp).astype(np.float64)
        if prec == gbe.PREC_FP64:
            T, k = np.ceil(m / 64), 16 * np.ceil(m / 16)
            want = np.sum(2 * 64 * 64 * k * T * (T + 1) / 2 / 1.2e6)
        else:
            T, nk = np.ceil(m / 128), np.ceil(m / 32)
            want = np.sum(T * (T + 1) / 2 * np.maximum(7.5, 0.6 * nk)) / ctx.sm_count
        np.testing.assert_allclose(cost[i], want, rtol=1e-12)
    assert best == int(np.argmin(cost))
    cc, sp, si = parts.export()
    cc2, sp2_, si2 = gbe.partition(ctx, G, gbe.PART_SPATIAL_CELLS, ncell=cands[best], site_struct=st).export()
    assert np.array_equal(cc, cc2) and np.array_equal(sp, sp2_) and np.array_equal(si, si2)
    print("partition costs:", dict(zip(cands, cost)), "best", cands[best])


@pytest.mark.parametrize("prec,tol", [(gbe.PREC_FP64, 1e-10), (gbe.PREC_FP16X6, 1e-6)])
def test_end_to_end_gpu_chain(ctx, prec, tol):
    """GPU H -> graph -> partition -> SP2 -> assembly against the oracle's own chain."""
    w = synth.lattice(8, seed=0)
    st = gbe.sites(torch.from_numpy(w["pos"]).cuda(), torch.from_numpy(w["onsite"]).cuda(), w["box"])
    Hgpu = gbe.build_hamiltonian(ctx, st)
    Hv = Hgpu.csr()
    G = gbe.build_graph(ctx, Hv, gbe.GRAPH_H2_THRESH, thresh=1e-5)
    Pg = gbe.partition(ctx, G, gbe.PART_SPATIAL_CELLS, ncell=(4, 4, 4), site_struct=st)
    Ho = hamiltonian.build_h(w["pos"], w["box"], w["onsite"])
    N = Ho.shape[0]
    subs_o, nc_o = partition.subgraphs(graph.h2_threshold(Ho, 1e-5),
                                       partition.spatial_cores(w["pos"], w["box"], (4, 4, 4)))
    subs_g, nc_g = export_parts(Pg)
    assert all(np.array_equal(a, b) for a, b in zip(subs_g, subs_o))
    _, logd = sp2.sp2_dense(Ho, N // 2)
    Dref = sp2.sp2_graph(Ho, subs_o, nc_o, N // 2, seq=logd.seq)[0].toarray()
    X, rep = gbe.sp2_submatrices(ctx, Hv, Pg, gbe.sp2_params(N // 2, prec=prec, seq=logd.seq))
    D, _, _ = assembled_dense(ctx, X, Pg, N)
    assert np.abs(D - Dref).max() <= tol
