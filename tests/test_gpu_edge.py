"""Degenerate and out-of-range inputs of the SP2 path, through the C ABI.

- Partitions that cannot be imported (no subgraph, an empty subgraph, no core vertex, an
  index outside H) are rejected on the host with GBE_EINVAL, before any device work.
- Singleton subgraphs (m_s = 1, every vertex its own core and no halo): the graph SP2
  reduces to the scalar recursion on each diagonal entry of X0, compared with the oracle.
- A subgraph whose dense rows exceed the gather's shared memory (more than 2432 vertices)
  has them staged in global memory: the 2600-site complete graph, FP64 and FP64TC, against
  the oracle's dense SP2.  One whose hash table exceeds it too (8193 vertices) is rejected
  with GBE_ECAPACITY before any kernel runs, and the context stays usable.
- A replayed branch sequence longer than n_max is rejected with GBE_EINVAL (it would be cut
  short without notice), and one of exactly n_max steps runs whole.
"""
import numpy as np
import pytest

from oracle import sp2

pytestmark = pytest.mark.gpu

from tests.gpu_helpers import assembled_dense, device_csr, gbe, import_parts, lattice_case, oracle_graph_sp2, torch  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    return gbe.Context(0)


def test_bad_partitions_rejected(ctx):
    lib = gbe.load_library()
    import ctypes
    def imp(n, cc, sp, si):
        cc = np.asarray(cc, np.int32); sp = np.asarray(sp, np.int64); si = np.asarray(si if len(si) else [0], np.int32)
        h = ctypes.c_void_p()
        return lib.gbe_parts_import(ctx.handle, n, len(cc), gbe._ptr(cc), gbe._ptr(sp), gbe._ptr(si), ctypes.byref(h))
    assert imp(4, [], [0], []) == gbe.GBE_EINVAL                 # no subgraph
    assert imp(0, [1], [0, 1], [0]) == gbe.GBE_EINVAL            # no vertex
    assert imp(4, [1, 1], [0, 2, 2], [0, 1]) == gbe.GBE_EINVAL   # empty subgraph
    assert imp(4, [0], [0, 2], [0, 1]) == gbe.GBE_EINVAL         # no core vertex
    assert imp(4, [3], [0, 2], [0, 1]) == gbe.GBE_EINVAL         # more cores than vertices
    assert imp(4, [1], [0, 2], [0, 4]) == gbe.GBE_EINVAL         # index outside H
    assert imp(4, [1], [0, 2], [-1, 0]) == gbe.GBE_EINVAL


@pytest.mark.parametrize("prec,tol", [(gbe.PREC_FP64, 1e-12), (gbe.PREC_FP16X6, 1e-6), (gbe.PREC_BF16X3, 2e-4),
                                      (gbe.PREC_FP64TC, 1e-12)])
def test_singleton_subgraphs(ctx, prec, tol):
    w, H, _, _, _ = lattice_case(6, seed=2)
    N = H.shape[0]
    subs = [np.array([i]) for i in range(N)]
    nc = np.ones(N, dtype=np.int32)
    _, logd = sp2.sp2_dense(H, N // 2)
    seq = logd.seq[:12]
    Dref, _, _ = oracle_graph_sp2(H, subs, nc, seq=seq)
    parts = import_parts(ctx, N, subs, nc)
    X, rep = gbe.sp2_submatrices(ctx, device_csr(H), parts, gbe.sp2_params(N // 2, prec=prec, seq=seq))
    assert rep["iters"] == len(seq)
    D, col, _ = assembled_dense(ctx, X, parts, N)
    assert col.shape[1] == 1 and np.array_equal(col[:, 0], np.arange(N))
    assert np.count_nonzero(D - np.diag(np.diag(D))) == 0
    assert np.abs(D - Dref).max() <= tol


@pytest.mark.parametrize("prec", [gbe.PREC_FP64, gbe.PREC_FP64TC])
def test_large_subgraph_rows_staged_in_global_memory(ctx, prec):
    import synth
    from oracle import hamiltonian
    w = synth.disordered(2600, seed=11)
    H = hamiltonian.build_h(w["pos"], w["box"], w["onsite"])
    N = H.shape[0]
    Xo, log = sp2.sp2_dense(H, N // 2, n_max=100)
    Xo = np.asarray(Xo.todense() if hasattr(Xo, "todense") else Xo)
    full = import_parts(ctx, N, [np.arange(N)], np.array([N]))
    seq = list(log.seq)
    X, rep = gbe.sp2_submatrices(ctx, device_csr(H), full, gbe.sp2_params(N // 2, prec=prec, seq=seq, n_max=len(seq)))
    assert rep["iters"] == len(seq) and rep["status"] == 0
    Dg, _, _ = assembled_dense(ctx, X, full, N)
    assert np.abs(Dg - Xo).max() < 1e-10


def test_oversized_subgraph_rejected(ctx):
    w, H, _, _, _ = lattice_case(21, seed=0, thr=0.15)
    N = H.shape[0]
    big = np.arange(8193)
    subs = [big] + [np.array([i]) for i in range(8193, N)]
    nc = np.array([8193] + [1] * (N - 8193), dtype=np.int32)
    parts = import_parts(ctx, N, subs, nc)
    Hd = device_csr(H)
    with pytest.raises(gbe.GbeError) as e:
        gbe.sp2_submatrices(ctx, Hd, parts, gbe.sp2_params(N // 2, prec=gbe.PREC_FP64, n_max=4))
    assert e.value.code == gbe.GBE_ECAPACITY
    # the context still works: a partition at the bound runs
    ok = [np.arange(8192)] + [np.array([i]) for i in range(8192, N)]
    nc2 = np.array([8192] + [1] * (N - 8192), dtype=np.int32)
    parts2 = import_parts(ctx, N, ok, nc2)
    X, rep = gbe.sp2_submatrices(ctx, Hd, parts2, gbe.sp2_params(N // 2, prec=gbe.PREC_FP16X6, seq=[1, 0]))
    assert rep["iters"] == 2 and rep["status"] == 0


def test_objects_outliving_their_context():
    """A context destroyed while its objects still hold device memory (as when Python's
    cycle collector finalises them in any order): the objects are freed afterwards without
    error, and a new context works."""
    w, H, _, subs, nc = lattice_case(6, seed=1, thr=1e-3, ncell=(3, 3, 3))
    N = H.shape[0]
    c1 = gbe.Context(0)
    parts = import_parts(c1, N, subs, nc)
    X, rep = gbe.sp2_submatrices(c1, device_csr(H), parts, gbe.sp2_params(N // 2, prec=gbe.PREC_FP16X6, seq=[1, 0, 1]))
    assert rep["iters"] == 3
    c1.close()
    X.close()
    parts.close()
    c2 = gbe.Context(0)
    parts2 = import_parts(c2, N, subs, nc)
    X2, rep2 = gbe.sp2_submatrices(c2, device_csr(H), parts2, gbe.sp2_params(N // 2, prec=gbe.PREC_FP16X6, seq=[1, 0, 1]))
    assert rep2["iters"] == 3 and rep2["t1"] == rep["t1"]
    X2.close()
    parts2.close()
    c2.close()


def test_device_wait_timeout_is_reported(ctx):
    """The tensor-core kernel's device-side waits are bounded.  With a wait budget far below
    the latency of an operand copy every CTA gives up, records GBE_ETIMEOUT, waits (about a
    second at most) for the copies and MMAs it already issued, frees its TMEM and returns;
    the run reports the error, the context stays usable, and a run with the default budget
    then gives the same D as before."""
    w, H, _, subs, nc = lattice_case(6, seed=1, thr=1e-3, ncell=(3, 3, 3))
    N = H.shape[0]
    parts = import_parts(ctx, N, subs, nc)
    Hd = device_csr(H)
    seq = [1, 0, 1]
    X, rep = gbe.sp2_submatrices(ctx, Hd, parts, gbe.sp2_params(N // 2, prec=gbe.PREC_FP16X6, seq=seq))
    D0, _, _ = assembled_dense(ctx, X, parts, N)
    with pytest.raises(gbe.GbeError) as e:
        gbe.sp2_submatrices(ctx, Hd, parts, gbe.sp2_params(N // 2, prec=gbe.PREC_FP16X6, seq=seq, timeout_ms=1e-5), X)
    assert e.value.code == gbe.GBE_ETIMEOUT
    X, rep = gbe.sp2_submatrices(ctx, Hd, parts, gbe.sp2_params(N // 2, prec=gbe.PREC_FP16X6, seq=seq), X)
    assert rep["status"] == 0 and rep["iters"] == len(seq)
    D1, _, _ = assembled_dense(ctx, X, parts, N)
    assert np.array_equal(D0, D1)


def test_replay_longer_than_n_max_rejected(ctx):
    w, H, _, subs, nc = lattice_case(6, seed=4, thr=1e-2, ncell=(3, 3, 3))
    N = H.shape[0]
    parts = import_parts(ctx, N, subs, nc)
    Hd = device_csr(H)
    seq = [1, 0, 1, 0, 1, 0]
    with pytest.raises(gbe.GbeError) as e:
        gbe.sp2_submatrices(ctx, Hd, parts, gbe.sp2_params(N // 2, prec=gbe.PREC_FP16X6, seq=seq, n_max=5))
    assert e.value.code == gbe.GBE_EINVAL and "n_max" in str(e.value)
    X, rep = gbe.sp2_submatrices(ctx, Hd, parts, gbe.sp2_params(N // 2, prec=gbe.PREC_FP16X6, seq=seq, n_max=6))
    assert rep["iters"] == 6 and rep["seq"] == seq and rep["stop"] == "replay"


def test_host_arrays_flagged_as_device_are_refused(ctx):
    """Host arrays passed with on_device = 1 (H to gbe_sp2_run, D to gbe_assemble_D) are
    refused with GBE_EINVAL before anything is enqueued; the context keeps working."""
    import ctypes

    from tests.gpu_helpers import host_csr
    w, H, S, subs, nc = lattice_case(6, seed=3, thr=1e-2, ncell=(3, 3, 3))
    N = H.shape[0]
    parts = import_parts(ctx, N, subs, nc)
    Hh = host_csr(H)
    lie = gbe.Csr(Hh.n, Hh.nnz, Hh.rowptr, Hh.col, Hh.val, 1)
    lie._keep = Hh
    prm = gbe.sp2_params(N // 2, prec=gbe.PREC_FP16X6)
    X = gbe.subs_create(ctx, parts, gbe.PREC_FP16X6)
    with pytest.raises(gbe.GbeError) as e:
        gbe.sp2_run(ctx, lie, parts, prm, X)
    assert e.value.code == gbe.GBE_EINVAL and "device memory" in str(e.value)
    Hd = device_csr(H)
    gbe.sp2_run(ctx, Hd, parts, prm, X)
    n, width = gbe.assemble_width(ctx, X, parts)
    colh = np.zeros((n, width), np.int32)
    valh = np.zeros((n, width), np.float64)
    e_lie = gbe.Ell(n, width, colh.ctypes.data, valh.ctypes.data, 1)
    code = gbe.load_library().gbe_assemble_D(ctx.handle, X.handle, parts.handle, 0.0, ctypes.byref(e_lie))
    assert code == gbe.GBE_EINVAL
    gbe.assemble_D(ctx, X, parts, colh, valh)
    cold = torch.empty((n, width), dtype=torch.int32, device="cuda")
    vald = torch.empty((n, width), dtype=torch.float64, device="cuda")
    gbe.assemble_D(ctx, X, parts, cold, vald)
    torch.cuda.synchronize()
    assert np.array_equal(colh, cold.cpu().numpy()) and np.array_equal(valh, vald.cpu().numpy())
    assert np.isfinite(valh).all()
