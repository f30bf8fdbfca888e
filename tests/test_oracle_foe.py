"""Pins for the oracle's finite-temperature Chebyshev expansion (Eq. 7)."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import exact, graph, hamiltonian, partition, sp2


def test_fermi_function_closed_form():
    e = np.array([-50.0, -1.0, 0.3, 0.3 + 1e-12, 2.0, 800.0])
    with np.errstate(over="ignore"):   # the textbook form overflows to 1/inf = 0 at e = 800
        naive = 1.0 / (np.exp(4.0 * (e - 0.3)) + 1.0)
    np.testing.assert_allclose(sp2.fermi(e, 4.0, 0.3), naive, rtol=1e-13, atol=1e-300)
    assert sp2.fermi(0.3, 4.0, 0.3) == 0.5


def test_coefficients_reproduce_known_series():
    # the interpolant of T_3 itself (f(e) = T_3((e - a) / b)) is exactly c_3 = 1
    eps = (-2.0, 6.0)
    a, b = 2.0, 4.0
    K = 2 * 9
    t = np.pi * (np.arange(K) + 0.5) / K
    f = np.cos(3 * t)
    n = np.arange(9)
    c = (2.0 / K) * (np.cos(np.outer(n, t)) @ f)
    c[0] *= 0.5
    ref = np.zeros(9); ref[3] = 1.0
    np.testing.assert_allclose(c, ref, atol=1e-14)
    # and the Fermi coefficients evaluate back to the Fermi function at the nodes' energies
    cf = sp2.fermi_chebyshev_coeffs(1.5, 1.0, eps, 200)
    e = np.linspace(-2.0, 6.0, 7)
    val = np.polynomial.chebyshev.chebval((e - a) / b, cf)
    np.testing.assert_allclose(val, sp2.fermi(e, 1.5, 1.0), atol=1e-12)


def test_clenshaw_equals_forward_sum():
    rng = np.random.default_rng(0)
    A = rng.normal(size=(30, 30)); A = (A + A.T) / 2
    x = A / (1.01 * np.abs(np.linalg.eigvalsh(A)).max())
    c = rng.normal(size=13)
    np.testing.assert_allclose(sp2.clenshaw_dense(x, c), sp2.chebyshev_dense(x, c), atol=1e-12)


def test_foe_complete_graph_equals_fermi_of_eigenvalues():
    w = synth.lattice(6, seed=2)
    H = hamiltonian.build_h(w["pos"], w["box"], w["onsite"])
    N = H.shape[0]
    ev, V = np.linalg.eigh(H.toarray())
    beta, mu = 3.0, 0.5 * (ev[N // 2 - 1] + ev[N // 2])
    ref = (V * sp2.fermi(ev, beta, mu)) @ V.T
    D, _ = sp2.foe_graph(H, [np.arange(N)], [N], beta, mu, 400)
    np.testing.assert_allclose(D.toarray(), ref, atol=1e-10)
    # high beta approaches the zero-temperature projector (gap 1.4 eV: the Fermi function at
    # the band edges differs from 0/1 by ~e^-20 at beta = 30)
    D0, _ = exact.density_matrix(H, N // 2)
    Dh, _ = sp2.foe_graph(H, [np.arange(N)], [N], 30.0, mu, 2000)
    assert np.abs(Dh.toarray() - D0).max() < 1e-8


def test_foe_graph_single_vertex_identity():
    # Eq. 6 with single-vertex cores: graph-partitioned = thresholded sparse expansion
    w = synth.lattice(4, seed=1)
    H = hamiltonian.build_h(w["pos"], w["box"], w["onsite"])
    N = H.shape[0]
    S = graph.h2_threshold(H, 1e-2)
    subs, nc = partition.subgraphs(S, partition.single_vertex_cores(N))
    eps = sp2.gershgorin(H)
    c = sp2.fermi_chebyshev_coeffs(2.0, 0.0, eps, 11)
    D, _ = sp2.foe_graph(H, subs, nc, 2.0, 0.0, 11, eps=eps, coeffs=c)
    a, b = 0.5 * (eps[1] + eps[0]), 0.5 * (eps[1] - eps[0])
    X = sp.csr_matrix((H - a * sp.identity(N)) / b)
    Pt = sp2.chebyshev_thresholded(X, S, c).toarray()
    np.testing.assert_allclose(D.toarray(), Pt, atol=1e-12)
