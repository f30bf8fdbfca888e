"""GPU parity of the QMD-like sequence (Sec. II.C): positions advance each step, H is rebuilt,
the graph comes from the previous step's thresholded D, and the SP2 branch sequence is fixed
before the step (the previous step's sequence, replayed), so the expansions exchange no
traces.  The whole chain (H, graph, partition, SP2, assembly) runs on the GPU in FP64 and is
compared with the oracle's chain step by step (graphs exact, D within 1e-10)."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import graph, hamiltonian, partition, sp2

pytestmark = pytest.mark.gpu

from tests.gpu_helpers import assembled_dense, gbe, torch  # noqa: E402

TAU = 1e-2          # graph from |D_prev| >= TAU
H2_FIRST = 0.15     # first step: |H^2| >= 0.15 (no previous D)
NCELL = (4, 4, 4)


def test_qmd_chain_matches_oracle():
    ctx = gbe.Context(0)
    w = synth.lattice(8, seed=0)
    N = w["pos"].shape[0]
    vel = synth.velocities(N, seed=1)
    D_prev_o = D_prev_g = None
    seq = None
    for t in range(4):
        pos = synth.advance(w["pos"], vel, w["box"], t)
        # oracle step
        H = hamiltonian.build_h(pos, w["box"], w["onsite"])
        S = graph.h2_threshold(H, H2_FIRST) if t == 0 else graph.d_threshold(D_prev_o, TAU)
        subs, nc = partition.subgraphs(S, partition.spatial_cores(pos, w["box"], NCELL))
        Do, log = sp2.sp2_graph(H, subs, nc, N // 2, seq=seq, n_max=60)
        # GPU step
        st = gbe.sites(torch.from_numpy(pos).cuda(), torch.from_numpy(w["onsite"]).cuda(), w["box"])
        Hg = gbe.build_hamiltonian(ctx, st)
        if t == 0:
            G = gbe.build_graph(ctx, Hg.csr(), gbe.GRAPH_H2_THRESH, thresh=H2_FIRST)
        else:
            G = gbe.build_graph(ctx, Hg.csr(), gbe.GRAPH_D_THRESH, thresh=TAU, D_prev=D_prev_g)
        parts = gbe.partition(ctx, G, gbe.PART_SPATIAL_CELLS, ncell=NCELL, site_struct=st)
        cc, sub_ptr, sub_idx = parts.export()
        assert list(cc) == list(nc)
        assert all(np.array_equal(a, b) for a, b in zip(np.split(sub_idx, sub_ptr[1:-1]), subs))
        X, rep = gbe.sp2_submatrices(ctx, Hg.csr(), parts,
                                     gbe.sp2_params(N // 2, prec=gbe.PREC_FP64, seq=seq, n_max=60))
        assert rep["seq"] == log.seq
        Dg, col, val = assembled_dense(ctx, X, parts, N)
        Do = Do.toarray()
        assert np.abs(Dg - Do).max() <= 1e-10
        # next step: graph from this D, sequence fixed in advance (this step's)
        D_prev_o = sp.csr_matrix(Do)
        D_prev_g = gbe.ell_struct(torch.from_numpy(col).cuda(), torch.from_numpy(val).cuda())
        seq = log.seq if seq is None else seq
