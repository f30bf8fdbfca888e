"""Pins for the oracle's graphs (brute-force dense patterns) and partitions."""
import numpy as np
import scipy.sparse as sp

import synth
from oracle import graph, hamiltonian, partition


def small_h(L=4, seed=1):
    w = synth.lattice(L, seed=seed)
    return w, hamiltonian.build_h(w["pos"], w["box"], w["onsite"])


def dense_pattern(G):
    return np.asarray(G.toarray(), dtype=bool)


def test_h2_threshold_brute_force():
    w = synth.disordered(150, seed=3)
    for H in (small_h()[1], hamiltonian.build_h(w["pos"], w["box"], w["onsite"])):
        Hd = H.toarray()
        H2 = Hd @ Hd
        for thr in (1e-5, 1e-2, 0.3):
            ref = (np.abs(H2) >= thr) | np.eye(len(Hd), dtype=bool)
            ref = ref | ref.T
            np.testing.assert_array_equal(dense_pattern(graph.h2_threshold(H, thr)), ref)
    # the disordered case has (H^2)_ij <= -thr entries, so a threshold on the signed value
    # rather than the magnitude (Eq. 2 reading) fails above
    assert (H2 <= -0.3).any()


def test_d_threshold_symmetrises():
    D = sp.csr_matrix(np.array([[0.5, 0.0, 0.2], [1e-6, 0.5, 0.0], [0.0, 0.0, 0.5]]))
    G = dense_pattern(graph.d_threshold(D, 1e-5))
    ref = np.array([[1, 0, 1], [0, 1, 0], [1, 0, 1]], dtype=bool)
    np.testing.assert_array_equal(G, ref)


def test_eq8_and_hk_brute_force():
    _, H = small_h(L=5)
    Hd = H.toarray()
    rng = np.random.default_rng(0)
    Dd = rng.normal(size=Hd.shape) * (rng.uniform(size=Hd.shape) < 0.05)
    A = ((np.abs(Dd) >= 0.5) | (np.abs(Dd.T) >= 0.5) | (Hd != 0) | np.eye(len(Hd), dtype=bool)).astype(int)
    ref = (A @ A) > 0
    np.testing.assert_array_equal(dense_pattern(graph.eq8_symbolic(sp.csr_matrix(Dd), H, 0.5)), ref)
    P = ((Hd != 0) | np.eye(len(Hd), dtype=bool)).astype(int)
    ref3 = (P @ P @ P) > 0
    np.testing.assert_array_equal(dense_pattern(graph.hk_pattern(H, 3)), ref3)
    # a 1-D chain, where the pattern of H^k is the band |i - j| <= k (closed form)
    n = 16
    T = sp.diags([np.ones(n - 1), np.ones(n), np.ones(n - 1)], [-1, 0, 1]).tocsr()
    band = np.abs(np.subtract.outer(np.arange(n), np.arange(n)))
    for k in (1, 2, 3, 5):
        np.testing.assert_array_equal(dense_pattern(graph.hk_pattern(T, k)), band <= k)


def test_cell_ids_closed_form():
    box = np.array([4.0, 4.0, 4.0])
    pos = np.array([[0.1, 0.1, 0.1], [3.9, 0.1, 0.1], [0.1, 3.9, 0.1], [0.1, 0.1, 3.9], [2.0, 2.0, 2.0]])
    np.testing.assert_array_equal(partition.cell_ids(pos, box, (2, 2, 2)), [0, 4, 2, 1, 7])


def test_lattice_cores_are_2x2x2_blocks():
    w = synth.lattice(8, seed=0)
    cores = partition.spatial_cores(w["pos"], w["box"], (4, 4, 4))
    assert len(cores) == 64 and all(len(c) == 8 for c in cores)
    # ideal site (i,j,k) has index (i*8+j)*8+k; sites sit 0.5a from cell walls, jitter is 0.05a
    ijk = np.stack(np.unravel_index(cores[0], (8, 8, 8)), 1)
    assert ijk.max() <= 1 and ijk.min() == 0


def test_halo_brute_force():
    _, H = small_h(L=6, seed=2)
    S = graph.h2_threshold(H, 1.0)
    Sd = dense_pattern(S)
    cores = partition.block_cores(H.shape[0], 7)
    subs, nc = partition.subgraphs(S, cores)
    # a sparse graph (about 34 of 216 neighbours per vertex): core members' neighbourhoods
    # differ, so a halo of one member alone, or of the wrong members, fails below
    assert max(len(idx) for idx in subs) < H.shape[0] // 2
    for C, idx, c in zip(cores, subs, nc):
        assert c == len(C)
        np.testing.assert_array_equal(idx[:c], C)
        halo = sorted(set(np.nonzero(Sd[C].any(0))[0]) - set(C))
        np.testing.assert_array_equal(idx[c:], halo)


def test_h2_threshold_rows_equals_full():
    w = synth.disordered(1200, seed=8)
    H = hamiltonian.build_h(w["pos"], w["box"], w["onsite"])
    full = graph.h2_threshold(H, 0.1).tocsr()
    rows = np.array([0, 5, 6, 400, 1199])
    part = graph.h2_threshold_rows(H, 0.1, rows)
    for i in rows:
        np.testing.assert_array_equal(part[i].indices, full[i].indices)
    others = np.setdiff1d(np.arange(1200), rows)
    assert part[others].nnz == 0
