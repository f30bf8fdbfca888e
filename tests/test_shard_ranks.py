"""Sharding one system's subgraphs over ranks (several GPUs; host logic on CPU).

The subgraph expansions are independent (Sec. II.A, after Eq. 6), so a run over R ranks
gives each rank a share of the subgraphs (gbe_shard_assign: greedy longest-processing-time
on m_s^3) and exchanges only the global traces that pick the branch (global-trace mode;
a pre-determined sequence needs none, Sec. II.C).  Each rank contributes its per-subgraph
trace sums at their global positions and zeros elsewhere, so the all-reduce is exact and
every rank decides exactly as one rank would.

Here: the assignment's properties, and a world-size-2 gloo run in which each rank squares
its own subgraphs (the oracle's dense products stand in for the GPU's squarings, which
have no CPU path) and exchanges its trace buffer through the binding's dist_exchange: the
branch sequence equals the one-rank oracle's and the union of the ranks' D columns equals
its D bit for bit.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import paper_1603_00937_gb300 as gbe  # noqa: E402


def _case():
    import synth
    from oracle import graph, hamiltonian, partition
    w = synth.disordered(512, seed=5)
    H = hamiltonian.build_h(w["pos"], w["box"], w["onsite"])
    S = graph.h2_threshold(H, 0.3)
    subs, nc = partition.subgraphs(S, partition.spatial_cores(w["pos"], w["box"], (3, 3, 3)))
    sub_ptr = np.concatenate([[0], np.cumsum([len(s) for s in subs])]).astype(np.int64)
    return H, subs, nc, sub_ptr


def test_assignment_is_balanced_greedy_and_deterministic():
    rng = np.random.default_rng(1)
    m = rng.integers(50, 700, size=97)
    sp = np.concatenate([[0], np.cumsum(m)]).astype(np.int64)
    cost = m.astype(float) ** 3
    for world in (1, 2, 3, 8):
        owner, load = gbe.shard_assign(sp, world)
        assert owner.min() >= 0 and owner.max() < world
        np.testing.assert_allclose([cost[owner == r].sum() for r in range(world)], load, rtol=1e-12)
        # the greedy bound of longest-processing-time: no rank exceeds the mean by more than one subgraph
        assert load.max() <= cost.sum() / world + cost.max() + 1e-6
        owner2, _ = gbe.shard_assign(sp, world)
        assert np.array_equal(owner, owner2)
    # largest first (ties: lower index), each to the least loaded rank (ties: lower rank):
    # sizes 10, 20, 20, 10 -> subgraph 1 to rank 0, 2 to rank 1, 0 to rank 0, 3 to rank 1
    owner, _ = gbe.shard_assign(np.array([0, 10, 30, 50, 60], np.int64), 2)
    assert list(owner) == [0, 0, 1, 1]
    # more ranks than subgraphs: the extra ranks own nothing
    owner, load = gbe.shard_assign(np.array([0, 5, 9], np.int64), 4)
    assert sorted(owner) == [0, 1] and load[2] == load[3] == 0.0


def _rank_run(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    from oracle import sp2
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        H, subs, nc, sub_ptr = _case()
        N, P = H.shape[0], len(subs)
        owner, _ = gbe.shard_assign(sub_ptr, world)
        mine = [g for g in range(P) if owner[g] == rank]
        eps = sp2.gershgorin(H)
        xs = sp2.gather_submatrices(H, [subs[g] for g in mine], eps)
        exch = gbe.dist_exchange()
        buf = np.zeros(2 * P + 1)
        log = sp2.Log()
        n = 0
        while True:
            Ss = [x @ x for x in xs]
            buf[:] = 0.0
            for x, s_, g in zip(xs, Ss, mine):
                c = nc[g]
                buf[g] = float(np.trace(x[:c, :c]))
                buf[P + g] = float(np.trace(s_[:c, :c]))
            exch(buf.ctypes.data, len(buf), None)
            assert buf[2 * P] == 0.0
            # global subgraph order, as the one-rank oracle adds them
            t1 = sum(float(v) for v in buf[:P])
            t2 = sum(float(v) for v in buf[P:2 * P])
            b = sp2._decide(log, n, t1, t2, N // 2, 1e-10, 10, 100, None)
            if b is None:
                break
            xs = [s_ if b else 2.0 * x - s_ for x, s_ in zip(xs, Ss)]
            log.seq.append(int(b))
            n += 1
        D = sp2.assemble(xs, [subs[g] for g in mine], [nc[g] for g in mine], N).tocoo()
        out[rank] = (list(log.seq), log.stop, D.row.copy(), D.col.copy(), D.data.copy(), len(mine))
    finally:
        dist.destroy_process_group()


def test_two_ranks_match_one_rank_bit_for_bit():
    from oracle import sp2
    import scipy.sparse as sps
    H, subs, nc, _ = _case()
    N = H.shape[0]
    Dref, logr = sp2.sp2_graph(H, subs, nc, N // 2)
    port = socket.socket()
    port.bind(("127.0.0.1", 0))
    p = port.getsockname()[1]
    port.close()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank_run, args=(r, 2, p, out)) for r in range(2)]
        for pr in procs:
            pr.start()
        for pr in procs:
            pr.join(300)
            assert pr.exitcode == 0
        res = dict(out)
    assert res[0][0] == res[1][0] == logr.seq and res[0][1] == logr.stop
    assert res[0][5] > 0 and res[1][5] > 0 and res[0][5] + res[1][5] == len(subs)
    D = sum(sps.coo_matrix((r[4], (r[2], r[3])), shape=(N, N)).tocsc() for r in res.values())
    diff = (D - Dref.tocsc()).tocoo()
    assert diff.nnz == 0 or np.abs(diff.data).max() == 0.0
