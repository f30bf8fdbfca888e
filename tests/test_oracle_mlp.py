"""Pins for the oracle's edge-classifier MLP: finite differences, closed forms, Adam."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import hamiltonian, mlp


def small_batch(n=40, seed=0):
    rng = np.random.default_rng(seed)
    F = rng.normal(size=(n, mlp.NF))
    y = (rng.uniform(size=n) < 0.4).astype(float)
    return F, y


def test_gradient_matches_central_differences():
    h = 8
    rng = np.random.default_rng(3)
    p = rng.normal(0, 0.5, mlp.n_params(h))
    F, y = small_batch()
    _, g = mlp.loss_and_grad(p, F, y, h=h, rounded=False)
    eps = 1e-6
    for k in rng.choice(len(p), 40, replace=False):
        d = np.zeros_like(p); d[k] = eps
        lp = mlp.bce_loss(mlp.forward(p + d, F, h, rounded=False), y)
        lm = mlp.bce_loss(mlp.forward(p - d, F, h, rounded=False), y)
        assert abs((lp - lm) / (2 * eps) - g[k]) < 1e-7 * max(1.0, abs(g[k]))


def test_bias_only_network_closed_form():
    h = 8
    p = np.zeros(mlp.n_params(h))
    p[-1] = 0.7                       # b3
    F, y = small_batch()
    z = mlp.forward(p, F, h, rounded=False)
    assert np.all(z == 0.7)
    loss, g = mlp.loss_and_grad(p, F, y, h=h, rounded=False)
    assert loss == pytest.approx(np.log1p(np.exp(0.7)) - 0.7 * y.mean(), rel=1e-14)
    assert g[-1] == pytest.approx(1 / (1 + np.exp(-0.7)) - y.mean(), rel=1e-14)
    assert np.all(g[:-1] == 0.0)
    assert mlp.bce_loss(np.zeros(5), np.array([0, 1, 0, 1, 1.0])) == pytest.approx(np.log(2.0), rel=1e-15)


def test_first_adam_step_is_sign_step():
    g = np.array([3.0, -2e-3, 0.5, -7.0])
    p, m, v = mlp.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=0.01, eps=0.0)
    np.testing.assert_allclose(p, -0.01 * np.sign(g), rtol=1e-12)


def test_fp16_rounding_of_weights():
    p = np.array([1.0 + 2 ** -11, 0.1, 65504.0], dtype=np.float32)
    r = mlp.fp16_round(p)
    assert r[0] == 1.0 and r[2] == 65504.0 and abs(r[1] - 0.1) < 1e-4


def test_rounded_network_uses_fp16_weights():
    """The default (rounded) forward pass and gradient are those of the network whose
    weights are the parameters rounded to IEEE half precision (numpy's float16 cast)."""
    h = 8
    rng = np.random.default_rng(6)
    p = rng.normal(0, 0.5, mlp.n_params(h))
    ph = p.astype(np.float16).astype(np.float64)
    assert np.any(ph != p)
    F, y = small_batch()
    np.testing.assert_array_equal(mlp.forward(p, F, h), mlp.forward(ph, F, h, rounded=False))
    assert np.abs(mlp.forward(p, F, h) - mlp.forward(p, F, h, rounded=False)).max() > 1e-6
    l1, g1 = mlp.loss_and_grad(p, F, y, h=h)
    l2, g2 = mlp.loss_and_grad(ph, F, y, h=h, rounded=False)
    assert l1 == l2
    np.testing.assert_array_equal(g1, g2)


def test_labels_threshold_the_magnitude():
    D = np.array([[0.5, -0.02, 1e-3], [0.01, 0.5, -1e-5], [0.0, 0.3, -0.5]])
    I = np.array([0, 0, 1, 1, 2, 2, 0])
    J = np.array([1, 2, 0, 2, 0, 1, 0])
    np.testing.assert_array_equal(mlp.labels(D, I, J, 1e-2), [1, 0, 1, 0, 0, 1, 1])
    np.testing.assert_array_equal(mlp.labels(sp.csr_matrix(D), I, J, 1e-5), [1, 1, 1, 1, 0, 1, 1])


def test_pairs_and_features_symmetric():
    w = synth.disordered(300, seed=4)
    H = hamiltonian.build_h(w["pos"], w["box"], w["onsite"])
    I, J, R = mlp.candidate_pairs(w["pos"], w["box"], 2.0)
    assert np.all(I != J) and np.all(R < 2.0)
    fwd = dict(zip(zip(I, J), range(len(I))))
    assert all((j, i) in fwd for i, j in zip(I, J))
    F = mlp.features(H, w["onsite"], I, J, R, 2.0)
    back = np.array([fwd[(j, i)] for i, j in zip(I, J)])
    np.testing.assert_allclose(F, F[back], rtol=1e-14, atol=0)
    # a pair inside the 2.5 a hopping range has its hopping as first feature
    k = np.argmin(R)
    assert F[k, 0] == pytest.approx(-np.log10(abs(H[I[k], J[k]])) / 12.0, rel=1e-12)


@pytest.mark.parametrize("rcand,count", [(1.5, 18), (1.9, 26), (2.1, 32), (2.3, 56)])
def test_candidate_pairs_simple_cubic_shells(rcand, count):
    # unjittered simple-cubic lattice: neighbour shells at 1, sqrt2, sqrt3, 2, sqrt5 hold
    # 6, 12, 8, 6, 24 sites
    w = synth.lattice(6, jitter=0.0)
    I, J, R = mlp.candidate_pairs(w["pos"], w["box"], rcand)
    assert np.all(np.bincount(I, minlength=216) == count)


def test_candidate_pairs_row_subset():
    w = synth.disordered(400, seed=9)
    I, J, R = mlp.candidate_pairs(w["pos"], w["box"], 2.2)
    rows = np.array([0, 17, 18, 250, 399])
    Is, Js, Rs = mlp.candidate_pairs(w["pos"], w["box"], 2.2, rows=rows)
    m = np.isin(I, rows)
    np.testing.assert_array_equal(Is, I[m])
    np.testing.assert_array_equal(Js, J[m])
    np.testing.assert_array_equal(Rs, R[m])


def test_graph_from_logits_limits_and_example():
    w = synth.disordered(300, seed=4)
    H = hamiltonian.build_h(w["pos"], w["box"], w["onsite"])
    I, J, R = mlp.candidate_pairs(w["pos"], w["box"], 3.0)
    z = np.linspace(-1.0, 1.0, len(I))
    # nothing kept: the pattern of H (which stores its diagonal)
    G = mlp.graph_from_logits(H, I, J, z, np.inf)
    assert (G != (H != 0)).nnz == 0
    # everything kept: the whole candidate ball (a superset of the 2.5 a hopping range)
    G = mlp.graph_from_logits(H, I, J, z, -np.inf)
    ball = np.zeros((300, 300), dtype=bool)
    ball[I, J] = True
    np.fill_diagonal(ball, True)
    np.testing.assert_array_equal(G.toarray(), ball)
    # a single kept pair (i, j) outside the hopping range adds both (i, j) and (j, i)
    k = int(np.argmax(R))
    zk = np.full(len(I), -5.0)
    zk[k] = 0.5
    G = mlp.graph_from_logits(H, I, J, zk, 0.0)
    extra = G.toarray() & ~(H != 0).toarray()
    assert set(zip(*np.nonzero(extra))) == {(I[k], J[k]), (J[k], I[k])}


def test_h2_feature_equals_matrix_square():
    # the row-dot-product form of (H^2)_ij against the explicit sparse product, and
    # against rows-only H (all other rows empty)
    w = synth.disordered(500, seed=11)
    H = hamiltonian.build_h(w["pos"], w["box"], w["onsite"])
    I, J, R = mlp.candidate_pairs(w["pos"], w["box"], 3.5, rows=np.arange(0, 500, 7))
    F = mlp.features(H, w["onsite"], I, J, R, 3.5)
    H2 = (H @ H).toarray()
    h2 = H2[I, J]
    np.testing.assert_allclose(F[:, 1], -np.log10(np.maximum(np.abs(h2), 1e-12)) / 12.0, rtol=1e-13, atol=1e-15)
    keep = np.union1d(I, J)
    Hr = sp.csr_matrix(H.toarray() * np.isin(np.arange(500), keep)[:, None])
    np.testing.assert_array_equal(mlp.features(Hr, w["onsite"], I, J, R, 3.5), F)
