"""Shared helpers of the GPU parity tests: build oracle inputs and call libgbe through the C ABI."""
import numpy as np
import pytest

import synth
from oracle import graph, hamiltonian, partition, sp2

torch = pytest.importorskip("torch")
import paper_1603_00937_gb300 as gbe  # noqa: E402


def device_csr(H):
    """Device gbe_csr of a scipy CSR matrix (int64 rowptr, int32 col, float64 val)."""
    H = H.tocsr()
    H.sort_indices()
    rp = torch.from_numpy(H.indptr.astype(np.int64)).cuda()
    ci = torch.from_numpy(H.indices.astype(np.int32)).cuda()
    va = torch.from_numpy(H.data.astype(np.float64)).cuda()
    return gbe.csr(H.shape[0], rp, ci, va)


def host_csr(H):
    H = H.tocsr()
    H.sort_indices()
    rp = np.ascontiguousarray(H.indptr.astype(np.int64))
    ci = np.ascontiguousarray(H.indices.astype(np.int32))
    va = np.ascontiguousarray(H.data.astype(np.float64))
    return gbe.csr(H.shape[0], rp, ci, va)


def import_parts(ctx, N, subs, nc):
    sub_ptr = np.zeros(len(subs) + 1, dtype=np.int64)
    sub_ptr[1:] = np.cumsum([len(s) for s in subs])
    return gbe.parts_import(ctx, N, np.asarray(nc, dtype=np.int32), sub_ptr, np.concatenate(subs).astype(np.int32))


def assembled_dense(ctx, X, parts, N, drop_tol=0.0):
    n, width = gbe.assemble_width(ctx, X, parts)
    col = torch.empty((n, width), dtype=torch.int32, device="cuda")
    val = torch.empty((n, width), dtype=torch.float64, device="cuda")
    gbe.assemble_D(ctx, X, parts, col, val, drop_tol)
    torch.cuda.synchronize()
    return gbe.ell_to_dense(col.cpu().numpy(), val.cpu().numpy(), N), col.cpu().numpy(), val.cpu().numpy()


def lattice_case(L=8, seed=0, thr=1e-5, ncell=None):
    w = synth.lattice(L, seed=seed)
    H = hamiltonian.build_h(w["pos"], w["box"], w["onsite"])
    S = graph.h2_threshold(H, thr)
    ncell = ncell or (L // 2,) * 3
    cores = partition.spatial_cores(w["pos"], w["box"], ncell)
    subs, nc = partition.subgraphs(S, cores)
    return w, H, S, subs, nc


def oracle_graph_sp2(H, subs, nc, seq=None, **kw):
    N = H.shape[0]
    D, log, xs = sp2.sp2_graph(H, subs, nc, N // 2, seq=seq, return_subs=True, **kw)
    return D.toarray(), log, xs


class _CudaArray:
    def __init__(self, ptr, count, typestr):
        self.__cuda_array_interface__ = {"shape": (int(count),), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3}


def device_array(ptr, count, typestr):
    """NumPy copy of `count` elements at a raw device pointer owned by libgbe."""
    torch.cuda.synchronize()
    return torch.as_tensor(_CudaArray(ptr, count, typestr), device="cuda").cpu().numpy().copy()
