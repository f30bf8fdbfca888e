"""Pins for the oracle's SP2 (dense, thresholded sparse, graph-partitioned, Chebyshev).

Each pin checks against something other than the oracle itself: closed forms, LAPACK
eigh, projector invariants, brute-force polynomial degrees, and the exact
column identity of Eq. (6) for serial (Krylov-type) expansions.
"""
import numpy as np
import numpy.polynomial.polynomial as npoly
import pytest
import scipy.sparse as sp

import synth
from oracle import exact, graph, hamiltonian, partition, sp2


def golden(name):
    """Values printed in the paper (tests/golden/paper_values.txt, each line cited there)."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_values.txt")
    for line in open(path):
        f = line.split()
        if f and f[0] == name:
            return [float(v) for v in f[1:]]
    raise KeyError(name)


@pytest.fixture(scope="module")
def c1():
    w = synth.lattice(8, seed=0)
    H = hamiltonian.build_h(w["pos"], w["box"], w["onsite"])
    return w, H


def test_gershgorin_tridiagonal_closed_form():
    n = 9
    T = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]).tocsr()
    # interior rows: 2 -/+ 2; end rows are inside that
    assert sp2.gershgorin(T) == (0.0, 4.0)


def test_gershgorin_encloses_spectrum(c1):
    _, H = c1
    lo, hi = sp2.gershgorin(H)
    w = np.linalg.eigvalsh(H.toarray())
    assert lo <= w[0] and w[-1] <= hi


def test_diagonal_h_gives_step_function():
    rng = np.random.default_rng(5)
    e = rng.permutation(np.linspace(-3.0, 2.0, 40))
    H = sp.diags(e).tocsr()
    D, log = sp2.sp2_dense(H, 13, idem_tol=1e-14)
    ref = np.diag((e <= np.sort(e)[12]).astype(float))
    np.testing.assert_allclose(D, ref, atol=1e-12)
    assert log.stop == "tol"


def test_dense_sp2_matches_eigh_and_projector_invariants(c1):
    _, H = c1
    N = H.shape[0]
    D, log = sp2.sp2_dense(H, N // 2)
    Dex, _ = exact.density_matrix(H, N // 2)
    assert np.abs(D - Dex).max() < 1e-12
    assert abs(np.trace(D) - N // 2) < 1e-10
    assert np.abs(D @ D - D).max() < 1e-12
    Hd = H.toarray()
    assert np.abs(Hd @ D - D @ Hd).max() < 1e-11
    assert 15 <= log.iters <= 40


def test_dimers_closed_form():
    """Decoupled dimers with onsite (e1, e2) and hopping t: each occupied bonding orbital
    (c, s) with tan(2 theta) = 2t/(e1 - e2) gives D_block = [[c^2, cs], [cs, s^2]]."""
    rng = np.random.default_rng(1)
    nd = 6
    blocks, refs = [], []
    for _ in range(nd):
        e1, e2, t = rng.uniform(-1, 1), rng.uniform(-1, 1), -rng.uniform(0.5, 1.5)
        h = np.array([[e1, t], [t, e2]])
        # lowest eigenvector of a 2x2 symmetric matrix, closed form
        lam = 0.5 * (e1 + e2) - np.sqrt(0.25 * (e1 - e2) ** 2 + t * t)
        v = np.array([t, lam - e1]); v /= np.linalg.norm(v)
        blocks.append(h); refs.append(np.outer(v, v))
    H = sp.block_diag([sp.csr_matrix(b) for b in blocks]).tocsr()
    Dref = sp.block_diag([sp.csr_matrix(r) for r in refs]).toarray()
    labels = np.repeat(np.arange(nd), 2)
    S = graph.complete_blocks(labels)
    cores = [np.array([2 * k, 2 * k + 1]) for k in range(nd)]
    subs, nc = partition.subgraphs(S, cores)
    D, log = sp2.sp2_graph(H, subs, nc, nd, idem_tol=1e-13)
    np.testing.assert_allclose(D.toarray(), Dref, atol=1e-12)
    Dd, _ = sp2.sp2_dense(H, nd, idem_tol=1e-13)
    np.testing.assert_allclose(Dd, Dref, atol=1e-12)


def test_expansion_order_doubles():
    """Each SP2 step is quadratic, so n steps give degree 2^n; the paper's 30 iterations
    give an order above one billion (Sec. II.B)."""
    p = np.array([0.0, 1.0])
    for n, b in enumerate([1, 0, 1, 1, 0, 0, 1, 0]):
        sq = npoly.polymul(p, p)
        p = sq if b else npoly.polysub(2 * np.pad(p, (0, len(sq) - len(p))), sq)
        assert len(np.trim_zeros(p, "b")) - 1 == 2 ** (n + 1)
    (iters,), (order,) = golden("sp2_iterations"), golden("sp2_min_order")
    assert 2 ** int(iters) > order


def test_complete_graph_equals_dense(c1):
    _, H = c1
    N = H.shape[0]
    S = graph.complete_blocks(np.zeros(N, dtype=int))
    cores = [np.arange(N)]
    subs, nc = partition.subgraphs(S, cores)
    D, log = sp2.sp2_graph(H, subs, nc, N // 2)
    Dd, logd = sp2.sp2_dense(H, N // 2)
    assert log.seq == logd.seq
    assert np.abs(D.toarray() - Dd).max() < 1e-13
    Xt, logt = sp2.sp2_thresholded(H, S, N // 2)
    assert logt.seq == logd.seq
    assert np.abs(Xt.toarray() - Dd).max() < 1e-13


def test_one_sp2_step_column_identity(c1):
    """One SP2 product: column i of floor(X0^2)_S equals column 0 of x[s_i]^2 (Eq. 6)."""
    _, H = c1
    S = graph.h2_threshold(H, 1e-3)
    eps = sp2.gershgorin(H)
    X0 = sp2.threshold_to(sp2.initial_x(H, eps), S)
    ref = sp2.threshold_to(X0 @ X0, S).toarray()
    subs, _ = partition.subgraphs(S, partition.single_vertex_cores(H.shape[0]))
    X0f = sp2.initial_x(H, eps)
    for i in range(0, H.shape[0], 37):
        idx = subs[i]
        x = X0f[idx][:, idx].toarray()
        col = np.zeros(H.shape[0]); col[idx] = (x @ x)[:, 0]
        np.testing.assert_allclose(col, ref[:, i], rtol=0, atol=1e-15)


@pytest.mark.parametrize("bit", [1, 0])
def test_thresholded_sp2_one_step_equals_graph_sp2(c1, bit):
    """O3 against O4 where Eq. 6 is exact: after one SP2 step (X^2 or 2X - X^2) the
    thresholded sparse iterate equals the assembly of single-vertex subgraph iterates, and
    the threshold bites (the unthresholded step has entries outside S)."""
    _, H = c1
    N = H.shape[0]
    S = graph.h2_threshold(H, 1e-3)
    subs, nc = partition.subgraphs(S, partition.single_vertex_cores(N))
    Xt, lt = sp2.sp2_thresholded(H, S, N // 2, seq=[bit])
    Dg, lg = sp2.sp2_graph(H, subs, nc, N // 2, seq=[bit])
    assert lt.seq == lg.seq == [bit]
    assert np.abs(Xt.toarray() - Dg.toarray()).max() < 1e-15
    X0 = sp2.initial_x(H, sp2.gershgorin(H)).toarray()
    full = X0 @ X0 if bit else 2 * X0 - X0 @ X0
    outside = ~S.toarray()
    assert np.abs(full[outside]).max() > 1e-6 and np.all(Xt.toarray()[outside] == 0.0)


def test_chebyshev_graph_identity(c1):
    """Eq. (6) is exact for serial expansions (Eqs. 1, 4, 5): thresholded sparse
    Chebyshev P_tau(X) equals the column assembly of per-vertex dense expansions."""
    _, H = c1
    lo, hi = sp2.gershgorin(H)
    X = ((H - 0.5 * (hi + lo) * sp.identity(H.shape[0])) / (0.5 * (hi - lo))).tocsr()
    S = graph.h2_threshold(H, 1e-4)
    coeffs = np.random.default_rng(2).normal(size=12)
    Pt = sp2.chebyshev_thresholded(X, S, coeffs).toarray()
    subs, _ = partition.subgraphs(S, partition.single_vertex_cores(H.shape[0]))
    Pg = sp2.chebyshev_graph(X, subs, coeffs).toarray()
    assert np.abs(Pt - Pg).max() < 1e-12
    # and the threshold actually bites: P_tau differs from the unthresholded P
    Pd = sp2.chebyshev_dense(X.toarray(), coeffs)
    assert np.abs(Pd - Pt).max() > 1e-6


def test_graph_sp2_error_falls_with_tau(c1):
    """Observation ii: accuracy improves as the threshold tau shrinks."""
    w, H = c1
    N = H.shape[0]
    Dex, _ = exact.density_matrix(H, N // 2)
    _, logd = sp2.sp2_dense(H, N // 2)
    cores = partition.spatial_cores(w["pos"], w["box"], (4, 4, 4))
    errs = []
    taus = sorted({t for t in golden("fig5_thresholds") if t >= 1e-2} | {3e-2}, reverse=True)
    assert taus == [1e-1, 3e-2, 1e-2]
    for tau in taus:
        S = graph.d_threshold(sp.csr_matrix(Dex), tau)
        subs, nc = partition.subgraphs(S, cores)
        D, _ = sp2.sp2_graph(H, subs, nc, N // 2, seq=logd.seq)
        errs.append(np.abs(D.toarray() - Dex).max())
    assert errs[0] > errs[1] > errs[2]


def test_graph_assembly_support_and_trace(c1):
    w, H = c1
    N = H.shape[0]
    S = graph.h2_threshold(H, 1e-5)
    cores = partition.spatial_cores(w["pos"], w["box"], (4, 4, 4))
    subs, nc = partition.subgraphs(S, cores)
    _, logd = sp2.sp2_dense(H, N // 2)
    D, log = sp2.sp2_graph(H, subs, nc, N // 2, seq=logd.seq)
    Dd = D.toarray()
    for idx, c in zip(subs, nc):
        outside = np.setdiff1d(np.arange(N), idx)
        assert np.all(Dd[np.ix_(outside, idx[:c])] == 0.0)
    # each truncated subgraph converges to its own projector (idempotent), while the
    # total core occupation only approximates N_occ (truncation, not a parity issue)
    assert abs(np.trace(Dd) - N // 2) < 0.5
    assert log.e[-1] < 1e-10


def test_graph_traces_are_core_traces(c1):
    """The cores partition the vertices, so the global traces of graph SP2 sum each
    subgraph's diagonal over its core positions only: at step 0 they are Tr X_0 and
    Tr X_0^2 of the whole matrix (each core's halo holds all its neighbours in H, so
    (x_s^2)_jj is the full row-times-column product)."""
    w, H = c1
    N = H.shape[0]
    S = graph.h2_threshold(H, 1e-5)
    cores = partition.spatial_cores(w["pos"], w["box"], (4, 4, 4))
    subs, nc = partition.subgraphs(S, cores)
    assert sum(nc) == N and max(len(s) for s in subs) < N
    lo, hi = sp2.gershgorin(H)
    X0 = (hi * np.eye(N) - H.toarray()) / (hi - lo)
    _, log = sp2.sp2_graph(H, subs, nc, N // 2, seq=[1])
    assert abs(log.t1[0] - np.trace(X0)) < 1e-11
    assert abs(log.t2[0] - np.sum(X0 * X0)) < 1e-11      # Tr X0^2 of a symmetric X0


def test_free_mode_stall_rule():
    log = sp2.Log()
    # e values fall then rise: stall must fire at the first n >= n_min with e_n >= e_{n-2}
    es = [1.0, 0.5, 0.25, 0.3, 0.6]
    out = [sp2._decide(log, n, 10.0 + e, 10.0, 10.0, 1e-12, 3, 50, None) for n, e in enumerate(es)]
    assert out[-1] is None and log.stop == "stall"
    assert all(o is not None for o in out[:-1])
