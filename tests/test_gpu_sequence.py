"""A pre-determined SP2 sequence (Sec. II.C) driving the GPU run.

The paper's MD run fixes the branch sequence of a step beforehand from a HOMO-LUMO gap
estimated at the previous step, so no trace is exchanged while the subgraphs are
squared.  Here, on the 8^3 lattice:
- a converged GPU run (the complete graph: one subgraph of every site, so the run reaches
  the two-level regime the estimate needs) gives its report to gbe_sp2_gap_estimate; the
  estimate lies inside the exact gap and agrees with the oracle's estimate from the
  oracle's own run to 1e-5 eV (the two runs' traces differ in their last bits, and the
  estimate reads them at a late step, where the idempotency error is ~1e-8, and maps them
  back through the inverse branch maps);
- gbe_sp2_sequence turns it into the branch sequence the oracle's sequence_from_gap gives
  for the same estimate, and as long as the oracle's sequence from its own estimate;
- the GPU replays that sequence on the complete graph (D against exact diagonalisation)
  and on the |H^2| > 1e-5 graph with cores of 8 (D against the oracle's graph SP2 replaying
  the same sequence), FP64 and FP64TC to 1e-10, FP16X6 to 1e-6.
"""
import numpy as np
import pytest

from oracle import exact, sp2

pytestmark = pytest.mark.gpu

from tests.gpu_helpers import assembled_dense, device_csr, gbe, import_parts, lattice_case, oracle_graph_sp2, torch  # noqa: E402

E_LO, E_HI, TOL_SEQ = 1e-8, 1e-3, 1e-12


@pytest.fixture(scope="module")
def case():
    w, H, S, subs, nc = lattice_case(8, seed=0, thr=1e-5)
    N = H.shape[0]
    eps = sp2.gershgorin(H)
    Dex, ev = exact.density_matrix(H, N // 2)
    _, logd = sp2.sp2_dense(H, N // 2, idem_tol=1e-11, n_max=80)
    ho, lo = sp2.gap_estimate(logd.t1, logd.t2, logd.seq, N // 2, eps, E_LO, E_HI)
    seq_o = sp2.sequence_from_gap(eps, ho, lo, TOL_SEQ)
    return dict(H=H, subs=subs, nc=nc, N=N, eps=eps, Dex=Dex, ev=ev, oracle_gap=(ho, lo), seq_o=seq_o)


@pytest.fixture(scope="module")
def ctx():
    return gbe.Context(0)


def gpu_sequence(ctx, case):
    N = case["N"]
    full = import_parts(ctx, N, [np.arange(N)], np.array([N]))
    _, rep = gbe.sp2_submatrices(ctx, device_csr(case["H"]), full,
                                 gbe.sp2_params(N // 2, prec=gbe.PREC_FP64, idem_tol=1e-11, n_max=80))
    assert rep["stop"] == "tol"
    homo, lumo = gbe.sp2_gap_estimate(rep, N // 2, E_LO, E_HI)
    return (homo, lumo), gbe.sp2_sequence(rep["eps"], homo, lumo, TOL_SEQ), full


def test_gap_estimate_and_sequence_from_a_gpu_run(ctx, case):
    (homo, lumo), seq, _ = gpu_sequence(ctx, case)
    ev, N = case["ev"], case["N"]
    assert ev[N // 2 - 1] <= homo < lumo <= ev[N // 2]
    np.testing.assert_allclose((homo, lumo), case["oracle_gap"], rtol=0, atol=1e-5)
    assert seq == sp2.sequence_from_gap(case["eps"], homo, lumo, TOL_SEQ)
    assert len(seq) == len(case["seq_o"])
    print(f"gap estimate [{homo:.6f}, {lumo:.6f}] eV (exact [{ev[N // 2 - 1]:.6f}, {ev[N // 2]:.6f}]), "
          f"{len(seq)} steps")


@pytest.mark.parametrize("prec,tol", [(gbe.PREC_FP64, 1e-10), (gbe.PREC_FP64TC, 1e-10), (gbe.PREC_FP16X6, 1e-6)])
def test_replayed_gap_sequence(ctx, case, prec, tol):
    _, seq, full = gpu_sequence(ctx, case)
    N, Hd = case["N"], device_csr(case["H"])
    # complete graph: the sequence converges the dense expansion to theta(mu - H)
    X, rep = gbe.sp2_submatrices(ctx, Hd, full, gbe.sp2_params(N // 2, prec=prec, seq=seq))
    assert rep["iters"] == len(seq) and rep["stop"] == "replay"
    D, _, _ = assembled_dense(ctx, X, full, N)
    err_ex = np.abs(D - case["Dex"]).max()
    # truncated graph: every subgraph follows the same pre-determined sequence
    parts = import_parts(ctx, N, case["subs"], case["nc"])
    X2, rep2 = gbe.sp2_submatrices(ctx, Hd, parts, gbe.sp2_params(N // 2, prec=prec, seq=seq))
    D2, _, _ = assembled_dense(ctx, X2, parts, N)
    Dref, _, _ = oracle_graph_sp2(case["H"], case["subs"], case["nc"], seq=seq)
    err_or = np.abs(D2 - Dref).max()
    print(f"prec {prec}: {len(seq)} steps, complete graph vs eigh {err_ex:.3e}, |H^2| graph vs oracle {err_or:.3e}")
    assert err_ex <= tol and err_or <= tol


@pytest.mark.parametrize("prec", [gbe.PREC_FP64, gbe.PREC_FP64TC])
def test_gap_from_previous_md_step(ctx, prec):
    """Sec. II.C's MD use: the gap estimated from one step's run fixes the next step's
    sequence.  The 8^3 lattice on its complete graph at t = 0 (free running), then the
    positions advanced by one step of seeded velocities: the sequence from the t = 0 estimate
    on the t = 1 Gershgorin bounds (from gbe_gershgorin_noalloc, passed to the run) gives D
    within 1e-10 of exact diagonalisation at t = 1, and the t = 1 run's own traces give the
    next estimate.  The estimate reads idempotency errors in [1e-6, 1e-2], above the
    FP64-grade tensor-core path's floor."""
    import synth
    from oracle import hamiltonian
    w = synth.lattice(8, seed=0)
    N = w["pos"].shape[0]
    vel = synth.velocities(N, seed=1)
    full = import_parts(ctx, N, [np.arange(N)], np.array([N]))

    def system(t):
        pos = synth.advance(w["pos"], vel, w["box"], t)
        return pos, hamiltonian.build_h(pos, w["box"], w["onsite"])

    _, H0 = system(0)
    _, rep0 = gbe.sp2_submatrices(ctx, device_csr(H0), full,
                                  gbe.sp2_params(N // 2, prec=prec, idem_tol=1e-11, n_max=80))
    gap = gbe.sp2_gap_estimate(rep0, N // 2, 1e-6, 1e-2)
    pos1, H1 = system(1)
    Hd = device_csr(H1)
    bounds = torch.empty(2, dtype=torch.float64, device="cuda")
    gbe.gershgorin_noalloc(ctx, Hd, bounds)
    eps = tuple(bounds.cpu().tolist())
    np.testing.assert_allclose(eps, sp2.gershgorin(H1), rtol=0, atol=1e-12)
    seq = gbe.sp2_sequence(eps, gap[0], gap[1], TOL_SEQ)
    X, rep1 = gbe.sp2_submatrices(ctx, Hd, full, gbe.sp2_params(N // 2, prec=prec, seq=seq, eps=eps,
                                                               n_max=len(seq)))
    assert rep1["iters"] == len(seq) and rep1["eps"] == eps
    D1, _, _ = assembled_dense(ctx, X, full, N)
    Dex, ev = exact.density_matrix(H1, N // 2)
    assert ev[N // 2 - 1] <= gap[0] < gap[1] <= ev[N // 2]
    assert np.abs(D1 - Dex).max() < 1e-10
    homo, lumo = gbe.sp2_gap_estimate(rep1, N // 2, 1e-6, 1e-2)
    assert ev[N // 2 - 1] <= homo < lumo <= ev[N // 2]
