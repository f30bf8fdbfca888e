"""Pre-determined SP2 sequences from a HOMO-LUMO gap (Sec. II.C): oracle pins, and the
library's host-only functions against the oracle (no GPU needed)."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import exact, hamiltonian, sp2


def diag_spectrum(seed=0, n=200, homo=-0.4, lumo=0.9):
    """Diagonal H: half the levels in [-6, homo] (HOMO exactly at homo), half in [lumo, 5]."""
    rng = np.random.default_rng(seed)
    occ = np.concatenate([[homo], rng.uniform(-6.0, homo, n // 2 - 1)])
    emp = np.concatenate([[lumo], rng.uniform(lumo, 5.0, n // 2 - 1)])
    return sp.diags(np.concatenate([occ, emp])).tocsr()


def test_gap_sequence_gives_step_function():
    H = diag_spectrum()
    eps = sp2.gershgorin(H)                       # exact for a diagonal matrix: (-6.., 5..)
    seq = sp2.sequence_from_gap(eps, -0.4, 0.9, 1e-13)
    X, log = sp2.sp2_dense(H, 100, seq=seq)
    d = np.diag(np.asarray(X.todense() if hasattr(X, "todense") else X))
    h = H.diagonal()
    np.testing.assert_allclose(d, (h <= -0.4).astype(float), atol=1e-12, rtol=0)


def test_gap_sequence_on_lattice_matches_eigh():
    w = synth.lattice(6, seed=1)
    H = hamiltonian.build_h(w["pos"], w["box"], w["onsite"])
    N = H.shape[0]
    D, ev = exact.density_matrix(H, N // 2)
    seq = sp2.sequence_from_gap(sp2.gershgorin(H), ev[N // 2 - 1], ev[N // 2], 1e-12)
    X, _ = sp2.sp2_dense(H, N // 2, seq=seq)
    X = np.asarray(X.todense() if hasattr(X, "todense") else X)
    assert np.abs(X - D).max() < 1e-10


def test_gap_estimate_exact_for_two_level_system():
    # every level but HOMO and LUMO sits at the spectral bounds, where SP2 is exact after one
    # step, so the two-level model holds exactly and the estimate recovers both levels
    levels = np.array([-3.0] * 5 + [-0.25] + [0.6] + [3.0] * 5)
    H = sp.diags(levels).tocsr()
    eps = (-3.0, 3.0)
    _, log = sp2.sp2_dense(H, 6, eps=eps)
    # (the window stays well above the trace rounding, ~1e-15, that late steps amplify)
    homo, lumo = sp2.gap_estimate(log.t1, log.t2, log.seq, 6, eps, 1e-5, 1e-1)
    assert homo == pytest.approx(-0.25, abs=1e-8) and lumo == pytest.approx(0.6, abs=1e-8)


def test_gap_estimate_is_conservative_on_lattice():
    w = synth.lattice(8, seed=0)
    H = hamiltonian.build_h(w["pos"], w["box"], w["onsite"])
    N = H.shape[0]
    _, ev = exact.density_matrix(H, N // 2)
    _, log = sp2.sp2_dense(H, N // 2)
    homo, lumo = sp2.gap_estimate(log.t1, log.t2, log.seq, N // 2, sp2.gershgorin(H), 1e-8, 1e-3)
    # the estimated gap lies inside the true one (other levels near the gap inflate the error)
    assert ev[N // 2 - 1] <= homo < lumo <= ev[N // 2]
    assert lumo - homo > 0.8 * (ev[N // 2] - ev[N // 2 - 1])


# ------------------------------------------------------------------ library host functions
gbe = pytest.importorskip("paper_1603_00937_gb300")


@pytest.fixture(scope="module")
def lib():
    import os
    if not os.path.exists(gbe.LIB_PATH):
        from paper_1603_00937_gb300 import build
        build.build()
    return gbe.load_library()


@pytest.mark.parametrize("homo,lumo,tol", [(-0.4, 0.9, 1e-12), (-0.1, 0.05, 1e-10), (2.0, 2.3, 1e-8)])
def test_library_sequence_matches_oracle(lib, homo, lumo, tol):
    eps = (-6.5, 5.5)
    assert gbe.sp2_sequence(eps, homo, lumo, tol) == sp2.sequence_from_gap(eps, homo, lumo, tol)


def test_library_sequence_errors(lib):
    with pytest.raises(gbe.GbeError) as e:
        gbe.sp2_sequence((-1.0, 1.0), 0.0, 1e-9, 1e-14, n_max=20)
    assert e.value.code == gbe.GBE_ENOCONV
    with pytest.raises(gbe.GbeError):
        gbe.sp2_sequence((-1.0, 1.0), 0.5, 0.2, 1e-10)


def test_library_gap_estimate_matches_oracle(lib):
    w = synth.lattice(8, seed=0)
    H = hamiltonian.build_h(w["pos"], w["box"], w["onsite"])
    N = H.shape[0]
    eps = sp2.gershgorin(H)
    _, log = sp2.sp2_dense(H, N // 2)
    rep = dict(iters=log.iters, eps=eps, seq=log.seq, t1=log.t1, t2=log.t2)
    ref = sp2.gap_estimate(log.t1, log.t2, log.seq, N // 2, eps, 1e-8, 1e-3)
    got = gbe.sp2_gap_estimate(rep, N // 2, 1e-8, 1e-3)
    # the oracle recovers x_l as a difference of two numbers near 1 (absolute rounding ~1e-16
    # on x_l ~ 1e-8 at the chosen step), the library from u = 1 - x directly: they agree to
    # that rounding mapped back to energies (~1e-9 eV over a 26 eV range)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-8)
    with pytest.raises(gbe.GbeError):
        gbe.sp2_gap_estimate(rep, N // 2, 1e-30, 1e-29)


@pytest.mark.parametrize("beta,mu,order", [(2.0, 0.0, 60), (10.0, -0.3, 400), (0.5, 1.2, 7)])
def test_library_fermi_coefficients_match_oracle(lib, beta, mu, order):
    eps = (-13.2, 12.9)
    np.testing.assert_allclose(gbe.fermi_coefficients(beta, mu, eps, order),
                               sp2.fermi_chebyshev_coeffs(beta, mu, eps, order), rtol=0, atol=1e-14)
