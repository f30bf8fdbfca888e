"""GPU parity of the finite-temperature Chebyshev expansion on subgraphs (Eq. 7 with Eq. 6).

FP64 path: within 1e-10 of the oracle's Clenshaw evaluation on the same graph and bounds.
FP16X6 path: every step adds the error of one split product, ~2^-34 representation plus
the FP32 accumulation of the second accumulator on the tensor cores, measured at 2-3e-10
of the iterates' scale B per step (they are stored divided by B); the recurrence is
stable (every tile of x b is computed as it is), so the errors add up over the order + 1
steps: bounded here by 2e-9 (order + 1) B.
"""
import numpy as np
import pytest

import synth
from oracle import hamiltonian, partition, sp2

pytestmark = pytest.mark.gpu

from tests.gpu_helpers import assembled_dense, device_csr, gbe, import_parts, lattice_case, torch  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    return gbe.Context(0)


@pytest.fixture(scope="module")
def case():
    w, H, S, subs, nc = lattice_case(8, seed=0, thr=1e-3, ncell=(4, 4, 4))
    beta, mu, order = 2.0, 0.0, 100
    D, c, xs = sp2.foe_graph(H, subs, nc, beta, mu, order, return_subs=True)
    return dict(H=H, subs=subs, nc=nc, beta=beta, mu=mu, order=order, D=D.toarray(), c=c)


@pytest.mark.parametrize("own_coeffs", [True, False])
def test_foe_fp64_parity(ctx, case, own_coeffs):
    H = case["H"]
    N = H.shape[0]
    parts = import_parts(ctx, N, case["subs"], case["nc"])
    X = gbe.subs_create(ctx, parts, gbe.PREC_FP64)
    rep = gbe.foe_run(ctx, device_csr(H), parts, X, case["beta"], case["mu"], case["order"], prec=gbe.PREC_FP64,
                      coeffs=None if own_coeffs else case["c"])
    assert rep["status"] == 0 and rep["order"] == case["order"] and rep["scale"] >= 1.0
    lo, hi = sp2.gershgorin(H)
    assert abs(rep["eps_min"] - lo) < 1e-12 and abs(rep["eps_max"] - hi) < 1e-12
    D, _, _ = assembled_dense(ctx, X, parts, N)
    err = np.abs(D - case["D"]).max()
    assert err <= 1e-10, err


def test_foe_fp16x6_bounded(ctx, case):
    H = case["H"]
    N = H.shape[0]
    parts = import_parts(ctx, N, case["subs"], case["nc"])
    X = gbe.subs_create(ctx, parts, gbe.PREC_FP16X6)
    rep = gbe.foe_run(ctx, device_csr(H), parts, X, case["beta"], case["mu"], case["order"], prec=gbe.PREC_FP16X6)
    assert rep["status"] == 0
    D, _, _ = assembled_dense(ctx, X, parts, N)
    err = np.abs(D - case["D"]).max()
    bound = 2e-9 * (case["order"] + 1) * rep["scale"]
    print(f"FOE FP16X6: max|dD| {err:.3e}, bound {bound:.3e}, scale B {rep['scale']:.3f}")
    assert err <= bound, (err, bound)
    # a second run on the same state reproduces the result bit for bit
    gbe.foe_run(ctx, device_csr(H), parts, X, case["beta"], case["mu"], case["order"], prec=gbe.PREC_FP16X6)
    D2, _, _ = assembled_dense(ctx, X, parts, N)
    np.testing.assert_array_equal(D2, D)


def test_foe_complete_graph_matches_fermi_of_eigenvalues(ctx):
    w = synth.lattice(6, seed=2)
    H = hamiltonian.build_h(w["pos"], w["box"], w["onsite"])
    N = H.shape[0]
    ev, V = np.linalg.eigh(H.toarray())
    beta, mu = 3.0, 0.5 * (ev[N // 2 - 1] + ev[N // 2])
    ref = (V * sp2.fermi(ev, beta, mu)) @ V.T
    parts = import_parts(ctx, N, [np.arange(N)], [N])
    X = gbe.subs_create(ctx, parts, gbe.PREC_FP64)
    gbe.foe_run(ctx, device_csr(H), parts, X, beta, mu, 400, prec=gbe.PREC_FP64)
    D, _, _ = assembled_dense(ctx, X, parts, N)
    assert np.abs(D - ref).max() <= 1e-9
