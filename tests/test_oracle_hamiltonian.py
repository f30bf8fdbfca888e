"""Pins for the oracle's tight-binding H (closed forms and lattice shell counts)."""
import numpy as np
import pytest

import synth
from oracle import hamiltonian


def two_sites(r, box=20.0):
    pos = np.array([[1.0, 1.0, 1.0], [1.0 + r, 1.0, 1.0]])
    return hamiltonian.build_h(pos, np.full(3, box), np.array([0.25, -0.75])).toarray()


def test_hopping_at_a_is_minus_one():
    H = two_sites(1.0)
    assert H[0, 1] == -1.0 and H[1, 0] == -1.0
    assert H[0, 0] == 0.25 and H[1, 1] == -0.75


def test_hopping_closed_forms():
    # r = 1.3a: -exp(-1);  r = sqrt(2) a: -exp(-(sqrt2 - 1)/0.3)
    assert two_sites(1.3)[0, 1] == pytest.approx(-0.367879441171442321595523770161, rel=1e-15)
    assert two_sites(np.sqrt(2.0))[0, 1] == pytest.approx(-0.251399524414250081216022781421, rel=1e-14)


def test_minimum_image_and_cutoff():
    box = np.full(3, 8.0)
    pos = np.array([[0.2, 4.0, 4.0], [7.7, 4.0, 4.0], [4.0, 4.0, 4.0], [6.49, 4.0, 4.0], [4.0, 6.51, 4.0]])
    H = hamiltonian.build_h(pos, box, np.zeros(5)).toarray()
    # 0 and 1 are 0.5 apart through the periodic boundary: -exp(5/3)
    assert H[0, 1] == pytest.approx(-5.2944900504700293668273720042, rel=1e-14)
    assert H[2, 3] != 0.0            # 2.49 a: inside the 2.5 a cutoff
    assert H[2, 4] == 0.0            # 2.51 a: outside
    np.testing.assert_array_equal(H, H.T)


def test_perfect_lattice_shell_count():
    # simple cubic shells inside 2.5a: 6 + 12 + 8 + 6 + 24 + 24 = 80 neighbours, plus the diagonal
    w = synth.lattice(6, jitter=0.0)
    H = hamiltonian.build_h(w["pos"], w["box"], w["onsite"])
    assert np.all(np.diff(H.indptr) == 81)
    d = H.diagonal()
    ijk = np.floor(w["pos"]).astype(int)
    np.testing.assert_array_equal(d, np.where(ijk.sum(1) % 2 == 0, 1.0, -1.0))


def test_rows_subset_matches_full():
    w = synth.lattice(5, seed=3)
    H = hamiltonian.build_h(w["pos"], w["box"], w["onsite"])
    rows = np.array([0, 17, 99, 124])
    Hr = hamiltonian.build_h(w["pos"], w["box"], w["onsite"], rows=rows)
    np.testing.assert_array_equal(Hr.toarray(), H[rows].toarray())


@pytest.mark.parametrize("kind", ["lattice", "disordered"])
def test_tree_build_equals_brute_force(kind):
    w = synth.lattice(10, seed=3) if kind == "lattice" else synth.disordered(3000, seed=5)
    Hb = hamiltonian.build_h(w["pos"], w["box"], w["onsite"])
    Ht = hamiltonian.build_h_tree(w["pos"], w["box"], w["onsite"])
    np.testing.assert_array_equal(Ht.indptr, Hb.indptr)
    np.testing.assert_array_equal(Ht.indices, Hb.indices)
    np.testing.assert_allclose(Ht.data, Hb.data, rtol=1e-15, atol=0)
