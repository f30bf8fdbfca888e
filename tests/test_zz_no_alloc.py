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
