"""Allocation-free Gershgorin bounds (gbe_gershgorin_noalloc) against the regular path.

Some callers cannot allocate device memory (their memory belongs to another allocator,
or they cannot accept the synchronisation an allocation may cause); for them the library
offers an entry point whose scratch is a fixed device array.  This file is named so that
pytest collects it last.
"""
import numpy as np
import pytest

import synth
from oracle import graph, hamiltonian, partition

pytestmark = pytest.mark.gpu

from tests.gpu_helpers import device_csr, gbe, import_parts, torch  # noqa: E402


def test_noalloc_bounds_match_regular_path_twice():
    ctx = gbe.Context(0, torch.cuda.current_stream().cuda_stream)
    w = synth.lattice(8, seed=11)
    H = hamiltonian.build_h(w["pos"], w["box"], w["onsite"])
    N = H.shape[0]
    Hd = device_csr(H)
    # regular path: the bounds gbe_sp2_run computes (reported by gbe_sp2_submatrices)
    subs, nc = partition.subgraphs(graph.h2_threshold(H, 1e-2), partition.spatial_cores(w["pos"], w["box"], (4, 4, 4)))
    parts = import_parts(ctx, N, subs, nc)
    _, rep = gbe.sp2_submatrices(ctx, Hd, parts, gbe.sp2_params(N // 2, prec=gbe.PREC_FP64, seq=[1, 0]))
    ref = np.array(rep["eps"])
    for _ in range(2):   # two calls in a row share the fixed scratch
        out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
        gbe.gershgorin_noalloc(ctx, Hd, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)


def test_noalloc_rejects_oversized_and_host_input():
    ctx = gbe.Context(0, torch.cuda.current_stream().cuda_stream)
    w = synth.lattice(6, seed=1)
    H = hamiltonian.build_h(w["pos"], w["box"], w["onsite"])
    Hd = device_csr(H)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    big = gbe.Csr(5_000_000, Hd.nnz, Hd.rowptr, Hd.col, Hd.val, 1)   # rejected before any launch
    with pytest.raises(gbe.GbeError) as e:
        gbe.gershgorin_noalloc(ctx, big, out)
    assert e.value.code == gbe.GBE_EINVAL and "4194304" in str(e.value)
    from tests.gpu_helpers import host_csr
    with pytest.raises(gbe.GbeError):
        gbe.gershgorin_noalloc(ctx, host_csr(H), out)


def test_noalloc_rejects_host_pointers_flagged_as_device():
    """bounds in host memory, or host CSR arrays passed with on_device = 1, are refused
    before anything is enqueued (a kernel would otherwise read or write the wrong memory)."""
    ctx = gbe.Context(0, torch.cuda.current_stream().cuda_stream)
    w = synth.lattice(6, seed=2)
    H = hamiltonian.build_h(w["pos"], w["box"], w["onsite"])
    Hd = device_csr(H)
    host_out = np.zeros(2)
    with pytest.raises(gbe.GbeError) as e:
        gbe.gershgorin_noalloc(ctx, Hd, host_out)
    assert e.value.code == gbe.GBE_EINVAL and "bounds" in str(e.value)
    from tests.gpu_helpers import host_csr
    Hh = host_csr(H)
    lie = gbe.Csr(Hh.n, Hh.nnz, Hh.rowptr, Hh.col, Hh.val, 1)
    lie._keep = Hh
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(gbe.GbeError) as e:
        gbe.gershgorin_noalloc(ctx, lie, out)
    assert e.value.code == gbe.GBE_EINVAL and "device memory" in str(e.value)
    # the context still works after the refusals
    gbe.gershgorin_noalloc(ctx, Hd, out)
    torch.cuda.synchronize()
    assert np.all(np.isfinite(out.cpu().numpy()))


def test_noalloc_nan_input_gives_nan_bounds_and_next_call_recovers():
    """A NaN in H makes both bounds NaN; the flag is cleared per call, so the next call on a
    clean H gives finite bounds again from the same scratch."""
    ctx = gbe.Context(0, torch.cuda.current_stream().cuda_stream)
    w = synth.lattice(6, seed=3)
    H = hamiltonian.build_h(w["pos"], w["box"], w["onsite"])
    bad = H.copy()
    bad.data = bad.data.copy()
    bad.data[len(bad.data) // 2] = np.nan
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    gbe.gershgorin_noalloc(ctx, device_csr(bad), out)
    torch.cuda.synchronize()
    assert np.all(np.isnan(out.cpu().numpy()))
    gbe.gershgorin_noalloc(ctx, device_csr(H), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    d = H.diagonal()
    off = np.asarray(abs(H).sum(axis=1)).ravel() - np.abs(d)
    np.testing.assert_allclose(got, [np.min(d - off), np.max(d + off)], rtol=0, atol=1e-12)
