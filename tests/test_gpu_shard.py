"""Sharded SP2 through the C ABI on one GPU: two ranks as two host threads.

Each thread has its own context and stream, owns the subgraphs gbe_shard_assign gives it
(gbe_parts_shard) and runs gbe_sp2_run with a trace exchange that meets the other thread
on the host (synchronise the stream, copy the buffer out, add the two buffers in rank
order, copy the sum back).  The threads' kernels never wait on each other; only the host
does.  Checked against one run of the whole partition on the same GPU:
- global-trace mode: the same branch sequence and traces bit for bit, and the union of
  the ranks' ELL rows equals the whole run's D bit for bit (FP64, FP16X6 and FP64TC);
- replay mode (a pre-determined sequence): no exchange is made, and D is again identical;
- a rank whose exchange fails makes both ranks return GBE_EPEER instead of hanging, and
  the contexts stay usable;
- the same independence on one GPU: gbe_sp2_replay_batched runs a replayed partition in
  batches that fit a memory budget, with D identical to one whole run.
"""
import threading

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from tests.gpu_helpers import device_csr, gbe, import_parts, lattice_case, torch  # noqa: E402

WORLD = 2


@pytest.fixture(scope="module")
def case():
    w, H, S, subs, nc = lattice_case(8, seed=0, thr=1e-2, ncell=(4, 4, 4))
    sub_ptr = np.concatenate([[0], np.cumsum([len(s) for s in subs])]).astype(np.int64)
    return dict(H=H, subs=subs, nc=nc, sub_ptr=sub_ptr, N=H.shape[0])


def whole_run(case, prec, seq=None):
    ctx = gbe.Context(0, torch.cuda.current_stream().cuda_stream)
    parts = import_parts(ctx, case["N"], case["subs"], case["nc"])
    Hd = device_csr(case["H"])
    X, rep = gbe.sp2_submatrices(ctx, Hd, parts, gbe.sp2_params(case["N"] // 2, prec=prec, seq=seq, n_max=60))
    n, width = gbe.assemble_width(ctx, X, parts)
    col = torch.empty((n, width), dtype=torch.int32, device="cuda")
    val = torch.empty((n, width), dtype=torch.float64, device="cuda")
    gbe.assemble_D(ctx, X, parts, col, val)
    torch.cuda.synchronize()
    return rep, col.cpu().numpy(), val.cpu().numpy()


def sharded_run(case, prec, seq=None, fail_rank=None, fail_call=3):
    N = case["N"]
    owner, _ = gbe.shard_assign(case["sub_ptr"], WORLD)
    streams = [torch.cuda.Stream() for _ in range(WORLD)]
    ctxs = [gbe.Context(0, s.cuda_stream) for s in streams]
    full = import_parts(ctxs[0], N, case["subs"], case["nc"])
    shards = [gbe.parts_shard(ctxs[r], full, owner, r) for r in range(WORLD)]
    Xs = [gbe.subs_create(ctxs[r], shards[r], prec) for r in range(WORLD)]
    Hd = device_csr(case["H"])
    width = max(len(s) for s in case["subs"])
    cols = [torch.empty((N, width), dtype=torch.int32, device="cuda") for _ in range(WORLD)]
    vals = [torch.empty((N, width), dtype=torch.float64, device="cuda") for _ in range(WORLD)]
    torch.cuda.synchronize()
    barrier = threading.Barrier(WORLD, timeout=10 if fail_rank is not None else 120)
    slots = [None] * WORLD
    calls = [0] * WORLD
    res = [None] * WORLD

    def exchange_of(r):
        def fn(ptr, count, stream):
            calls[r] += 1
            if r == fail_rank and calls[r] == fail_call:
                raise RuntimeError("planted exchange failure")
            torch.cuda.ExternalStream(stream).synchronize()
            t = torch.as_tensor(_View(ptr, count), device="cuda")
            slots[r] = t.cpu().numpy().copy()
            barrier.wait()
            total = slots[0].copy()
            for k in range(1, WORLD):
                total = total + slots[k]
            barrier.wait()
            t.copy_(torch.from_numpy(total))
            torch.cuda.current_stream().synchronize()
        return fn

    def rank_main(r):
        try:
            with torch.cuda.stream(streams[r]):
                prm = gbe.sp2_params(N // 2, prec=prec, seq=seq, n_max=60, exchange=exchange_of(r))
                gbe.sp2_run(ctxs[r], Hd, shards[r], prm, Xs[r])
                rep = gbe.sp2_report_get(ctxs[r], Xs[r]).as_dict()
                gbe.assemble_D(ctxs[r], Xs[r], shards[r], cols[r], vals[r])
                streams[r].synchronize()
                res[r] = ("ok", rep)
        except gbe.GbeError as e:
            res[r] = ("err", e.code)
            try:
                barrier.abort()
            except Exception:
                pass

    ths = [threading.Thread(target=rank_main, args=(r,)) for r in range(WORLD)]
    for t in ths:
        t.start()
    for t in ths:
        t.join(300)
        assert not t.is_alive()
    torch.cuda.synchronize()
    out = dict(res=res, calls=calls, owner=owner, ctxs=ctxs, shards=shards, Xs=Xs, Hd=Hd)
    if all(r[0] == "ok" for r in res):
        col = np.full((N, width), -1, np.int32)
        val = np.zeros((N, width))
        for r in range(WORLD):
            c, v = cols[r].cpu().numpy(), vals[r].cpu().numpy()
            own = c[:, 0] >= 0
            col[own], val[own] = c[own], v[own]
        out.update(col=col, val=val)
    return out


class _View:
    def __init__(self, ptr, count):
        self.__cuda_array_interface__ = {"shape": (int(count),), "typestr": "<f8", "data": (int(ptr), False),
                                         "version": 3}


@pytest.mark.parametrize("prec", [gbe.PREC_FP64, gbe.PREC_FP16X6, gbe.PREC_FP64TC])
def test_global_trace_shards_match_whole_run(case, prec):
    rep, col, val = whole_run(case, prec)
    out = sharded_run(case, prec)
    assert all(r[0] == "ok" for r in out["res"]), out["res"]
    assert len(set(out["owner"])) == WORLD
    for _, r in out["res"]:
        assert r["seq"] == rep["seq"] and r["stop"] == rep["stop"]
        assert r["t1"] == rep["t1"] and r["t2"] == rep["t2"]
    # one exchange after the gather and one per step, the same number on both ranks
    assert out["calls"][0] == out["calls"][1] == rep["iters"] + 1
    w = col.shape[1]
    assert np.array_equal(out["col"][:, :w], col) and np.all(out["col"][:, w:] == -1)
    assert np.array_equal(out["val"][:, :w], val)
    print(f"prec {prec}: {rep['iters']} steps ({rep['stop']}), shards of {np.bincount(out['owner'])} subgraphs")


def test_replay_shards_exchange_nothing(case):
    rep, col, val = whole_run(case, gbe.PREC_FP16X6)
    seq = rep["seq"]
    rep2, col2, val2 = whole_run(case, gbe.PREC_FP16X6, seq=seq)
    out = sharded_run(case, gbe.PREC_FP16X6, seq=seq)
    assert all(r[0] == "ok" for r in out["res"]) and out["calls"] == [0, 0]
    for _, r in out["res"]:
        assert r["seq"] == seq and r["stop"] == "replay"
    w = col2.shape[1]
    assert np.array_equal(out["col"][:, :w], col2) and np.array_equal(out["val"][:, :w], val2)


def test_failed_exchange_stops_both_ranks(case):
    out = sharded_run(case, gbe.PREC_FP64, fail_rank=1, fail_call=3)
    assert [r[0] for r in out["res"]] == ["err", "err"]
    assert all(r[1] == gbe.GBE_EPEER for r in out["res"])
    # the contexts still work: a replay run on a shard needs no exchange
    ctx, sh, X = out["ctxs"][0], out["shards"][0], out["Xs"][0]
    gbe.sp2_run(ctx, out["Hd"], sh, gbe.sp2_params(case["N"] // 2, prec=gbe.PREC_FP64, seq=[1, 0, 1]), X)
    r = gbe.sp2_report_get(ctx, X).as_dict()
    assert r["status"] == gbe.GBE_OK and r["iters"] == 3


@pytest.mark.parametrize("prec", [gbe.PREC_FP64, gbe.PREC_FP16X6, gbe.PREC_FP64TC])
def test_replay_in_batches_matches_whole_run(case, prec):
    """gbe_sp2_replay_batched: a partition replayed in batches of subgraphs whose iterates
    fit a budget (here a quarter of the whole, so at least four batches) gives, row for row,
    the D of one run over the whole partition with the same sequence, into device and host
    ELL buffers; a global-trace run and a budget below one subgraph's iterates are refused."""
    rep, _, _ = whole_run(case, prec)
    seq = rep["seq"]
    _, col2, val2 = whole_run(case, prec, seq=seq)
    ctx = gbe.Context(0, torch.cuda.current_stream().cuda_stream)
    parts = import_parts(ctx, case["N"], case["subs"], case["nc"])
    Hd = device_csr(case["H"])
    mpad = [(len(s) + 127) // 128 * 128 for s in case["subs"]]
    per = {gbe.PREC_FP64: 16, gbe.PREC_FP16X6: 16, gbe.PREC_FP64TC: 40}[prec]
    need = sum(p * p * per for p in mpad)
    prm = gbe.sp2_params(case["N"] // 2, prec=prec, seq=seq, n_max=len(seq))
    n, width = col2.shape
    col = torch.empty((n, width), dtype=torch.int32, device="cuda")
    val = torch.empty((n, width), dtype=torch.float64, device="cuda")
    nb = gbe.sp2_replay_batched(ctx, Hd, parts, prm, need // 4, col, val)
    assert nb >= 4
    assert np.array_equal(col.cpu().numpy(), col2) and np.array_equal(val.cpu().numpy(), val2)
    colh = np.empty((n, width), np.int32)
    valh = np.empty((n, width), np.float64)
    assert gbe.sp2_replay_batched(ctx, Hd, parts, prm, need, colh, valh) == 1
    assert np.array_equal(colh, col2) and np.array_equal(valh, val2)
    with pytest.raises(gbe.GbeError) as e:
        gbe.sp2_replay_batched(ctx, Hd, parts, gbe.sp2_params(case["N"] // 2, prec=prec), need, col, val)
    assert e.value.code == gbe.GBE_EINVAL
    with pytest.raises(gbe.GbeError) as e:
        gbe.sp2_replay_batched(ctx, Hd, parts, prm, min(mpad) ** 2 * per - 1, col, val)
    assert e.value.code == gbe.GBE_ECAPACITY


def test_replay_in_batches_reports_a_non_finite_H(case):
    """A NaN entry of H (found by the Gershgorin pass of the first batch) comes back from
    gbe_sp2_replay_batched as GBE_ENUMERIC, as it does from gbe_sp2_submatrices."""
    rep, _, _ = whole_run(case, gbe.PREC_FP16X6)
    seq = rep["seq"]
    ctx = gbe.Context(0, torch.cuda.current_stream().cuda_stream)
    parts = import_parts(ctx, case["N"], case["subs"], case["nc"])
    bad = case["H"].tocsr().copy()
    bad.sort_indices()
    bad.data[len(bad.data) // 3] = np.nan
    Hd = device_csr(bad)
    prm = gbe.sp2_params(case["N"] // 2, prec=gbe.PREC_FP16X6, seq=seq, n_max=len(seq))
    with pytest.raises(gbe.GbeError) as e:
        gbe.sp2_submatrices(ctx, Hd, parts, prm)
    assert e.value.code == gbe.GBE_ENUMERIC
    n = case["N"]
    width = max(len(s) for s in case["subs"])
    col = torch.empty((n, width), dtype=torch.int32, device="cuda")
    val = torch.empty((n, width), dtype=torch.float64, device="cuda")
    with pytest.raises(gbe.GbeError) as e:
        gbe.sp2_replay_batched(ctx, Hd, parts, prm, 1 << 40, col, val)
    assert e.value.code == gbe.GBE_ENUMERIC
