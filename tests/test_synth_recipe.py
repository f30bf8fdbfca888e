"""The seeded input generators follow the stated recipe (CPU).

Both the oracle and the CUDA path take their inputs from `synth`, so a drift in a
generator (a wrong jitter width, a density off by a factor, a species imbalance, an
unwrapped coordinate) would move every workload away from its stated shape without
any parity test noticing.  These checks hold the generators to the recipe: exact
properties exactly, distributions within several standard errors of the stated
parameters (deterministic seeds, so the checks do not flake).
"""
import numpy as np
import pytest

import synth


def _dev_from_centres(w):
    """Minimum-image displacement of each lattice site from its cell centre (i + 1/2) a."""
    L, a = w["L"], w["a"]
    g = np.arange(L)
    ijk = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    d = w["pos"] - (ijk + 0.5) * a
    return d - w["box"] * np.round(d / w["box"])


@pytest.mark.parametrize("L", [5, 16])
def test_lattice_exact_properties(L):
    w = synth.lattice(L, seed=0)
    N = L ** 3
    assert w["pos"].shape == (N, 3) and w["pos"].dtype == np.float64 and w["pos"].flags.c_contiguous
    assert np.all(w["box"] == L) and np.all(w["pos"] >= 0) and np.all(w["pos"] < w["box"])
    # rock-salt onsite pattern: +1 on i+j+k even, -1 on odd; nearest neighbours alternate
    i, j, k = np.unravel_index(np.arange(N), (L, L, L))
    np.testing.assert_array_equal(w["onsite"], np.where((i + j + k) % 2 == 0, 1.0, -1.0))
    assert w["onsite"].sum() == (0.0 if L % 2 == 0 else 1.0)
    # without jitter every site sits exactly on its cell centre
    w0 = synth.lattice(L, jitter=0.0)
    np.testing.assert_array_equal(_dev_from_centres(w0), 0.0)


def test_lattice_jitter_distribution():
    w = synth.lattice(16, seed=0)
    d = _dev_from_centres(w).ravel()          # 12288 draws of N(0, 0.05)
    se = 0.05 / np.sqrt(d.size)
    assert abs(d.mean()) < 5 * se
    assert abs(d.std() - 0.05) < 5 * 0.05 / np.sqrt(2 * d.size)
    assert np.abs(d).max() < 0.05 * 6         # no site leaves its cell: cores of whole blocks hold
    # the three axes are drawn independently
    c = np.corrcoef(_dev_from_centres(w).T)
    assert np.abs(c - np.eye(3)).max() < 5 / np.sqrt(w["pos"].shape[0])


def test_lattice_seeds():
    a, b, c = synth.lattice(6, seed=0), synth.lattice(6, seed=0), synth.lattice(6, seed=1)
    np.testing.assert_array_equal(a["pos"], b["pos"])
    assert not np.array_equal(a["pos"], c["pos"])
    np.testing.assert_array_equal(a["onsite"], c["onsite"])   # the onsite pattern draws nothing


@pytest.mark.parametrize("N,side", [(4096, 16.0), (131072, 50.8), (1048576, 101.6)])
def test_disordered_box_side(N, side):
    """Density 1/a^3: the box sides the workloads quote (16a, 50.8a, 101.6a)."""
    rho = 1.0
    s = (N / rho) ** (1.0 / 3.0)
    assert abs(s - side) < 0.05
    if N <= 131072:
        w = synth.disordered(N, seed=0)
        assert np.all(w["box"] == s)
        assert N / np.prod(w["box"]) == pytest.approx(1.0, rel=1e-12)


def test_disordered_distributions():
    N = 131072
    w = synth.disordered(N, seed=0)
    pos, box, sp, on = w["pos"], w["box"], w["species"], w["onsite"]
    assert pos.shape == (N, 3) and np.all(pos >= 0) and np.all(pos < box)
    # uniform: per-axis mean side/2 and variance side^2/12; octant counts N/8
    side = box[0]
    se = side / np.sqrt(12 * N)
    assert np.all(np.abs(pos.mean(axis=0) - side / 2) < 5 * se)
    assert np.all(np.abs(pos.var(axis=0) / (side ** 2 / 12) - 1) < 5 * np.sqrt(0.8 / N))
    octant = ((pos >= side / 2) * np.array([1, 2, 4])).sum(axis=1)
    counts = np.bincount(octant, minlength=8)
    chi2 = ((counts - N / 8) ** 2 / (N / 8)).sum()
    assert chi2 < 30                           # 7 degrees of freedom; P(chi2 > 30) ~ 1e-4
    # species 50/50, onsite N(+1, 0.1) for species 0 and N(-1, 0.1) for species 1
    assert set(np.unique(sp)) == {0, 1}
    n0 = int((sp == 0).sum())
    assert abs(n0 - N / 2) < 5 * np.sqrt(N / 4)
    for s, mu in ((0, 1.0), (1, -1.0)):
        x = on[sp == s]
        assert abs(x.mean() - mu) < 5 * 0.1 / np.sqrt(x.size)
        assert abs(x.std() - 0.1) < 5 * 0.1 / np.sqrt(2 * x.size)
    # the two species' onsite bands do not overlap at 10 sigma
    assert on[sp == 0].min() > 0 and on[sp == 1].max() < 0


def test_velocities_and_advance():
    N = 32768
    v = synth.velocities(N, seed=1)
    assert v.shape == (N, 3)
    assert np.all(np.abs(v.mean(axis=0)) < 5 * 0.01 / np.sqrt(N))
    assert np.all(np.abs(v.std(axis=0) - 0.01) < 5 * 0.01 / np.sqrt(2 * N))
    np.testing.assert_array_equal(v, synth.velocities(N, seed=1))
    w = synth.lattice(32, seed=0)
    for steps in (3, 100):
        p = synth.advance(w["pos"], v, w["box"], steps=steps)
        assert np.all(p >= 0) and np.all(p < w["box"])
        d = p - (w["pos"] + steps * v)
        # the only change besides the displacement is a whole-box wrap
        np.testing.assert_allclose(d / w["box"], np.round(d / w["box"]), atol=1e-12)
    # after 100 steps (displacement std 1a) sites at the faces have wrapped across them
    assert np.any(np.abs(d) > 1.0)


def test_advance_equals_the_plain_remainder():
    """synth.advance's masked wrap gives np.mod's bits: on lattices over short and long runs
    (the long ones take the np.mod path), and on values at 0, just below the box length, with
    denormal steps and with steps that land a hair below 0 (fl(y + b) rounds to b there)."""
    def plain(pos, vel, box, steps):
        p = np.mod(pos + steps * vel, box)
        p -= box * (p >= box)
        return p
    for L in (4, 8, 32):
        w = synth.lattice(L, seed=L)
        v = synth.velocities(w["pos"].shape[0], seed=L + 1)
        for steps in (0, 1, 3, 17, 64, 300, 5000, 100000):
            a = synth.advance(w["pos"], v, w["box"], steps)
            assert np.array_equal(a, plain(w["pos"], v, w["box"], steps))
            assert np.all(a >= 0) and np.all(a < w["box"])
    rng = np.random.default_rng(0)
    box = np.array([10.0, 10.0, 10.0])
    p0 = rng.uniform(0, 10, (20000, 3))
    v0 = rng.choice([-1.0, 1.0], (20000, 3)) * rng.uniform(0, 1e-3, (20000, 3))
    p0[:100] = 0.0
    p0[100:200] = np.nextafter(10.0, 0.0)
    v0[:50] = -1e-300
    v0[50:100] = -5e-324
    v0[200:300] = -(p0[200:300] + 1e-17)
    for steps in (1, 2, 7):
        a = synth.advance(p0, v0, box, steps)
        assert np.array_equal(a, plain(p0, v0, box, steps))
        assert np.all(a >= 0) and np.all(a < box)
    # a non-cubic box takes the plain path
    box2 = np.array([10.0, 12.0, 14.0])
    assert np.array_equal(synth.advance(p0, v0, box2, 3), plain(p0, v0, box2, 3))
