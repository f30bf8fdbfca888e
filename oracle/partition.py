"""Cores (communities) and core+halo subgraphs (oracle side).

Sec. II.A: the subgraph of a core vertex i holds i and every halo vertex directly
connected to i in S_tau (Fig. 1); observation vi generalises a core to a community of
vertices, whose subgraph is the core set plus all vertices adjacent to any core vertex.

Cores here are spatial cells (the paper's METIS partitioning is not available):
cell(x) = floor(x / box * ncell) per axis, linear id (cx * ny + cy) * nz + cz.  Cores
are listed in ascending cell id (empty cells skipped), core sites ascending; the halo
of a core set is the sorted union of its members' neighbours minus the core set; the
subgraph's local index list is core sites followed by halo sites.
"""
import numpy as np
import scipy.sparse as sp


def cell_ids(pos, box, ncell):
    """Linear spatial-cell id of each site (cores stand in for the graph partitioning of
    Sec. II.B, obs. vi-vii)."""
    ncell = np.asarray(ncell, dtype=np.int64)
    c = np.floor(pos / box * ncell).astype(np.int64)
    c = np.minimum(np.maximum(c, 0), ncell - 1)
    return (c[:, 0] * ncell[1] + c[:, 1]) * ncell[2] + c[:, 2]


def spatial_cores(pos, box, ncell):
    """Cores as spatial cells (communities of obs. vi standing in for the METIS partitioning of
    Sec. II.B): int64 arrays (ascending sites), one per non-empty cell in cell-id order."""
    cid = cell_ids(pos, box, ncell)
    order = np.argsort(cid, kind="stable")
    cs = cid[order]
    bounds = np.nonzero(np.diff(cs))[0] + 1
    return [np.sort(g) for g in np.split(order, bounds)]


def block_cores(N, core_size):
    """Cores as consecutive index blocks of core_size vertices (last one ragged; communities of
    obs. vi)."""
    return [np.arange(s, min(s + core_size, N)) for s in range(0, N, core_size)]


def subgraphs(S, cores):
    """Core+halo subgraphs (Sec. II.A, Fig. 1, obs. vi): each core set followed by the sorted
    vertices adjacent to it in S outside it.  Returns (sub_idx list, core counts)."""
    S = sp.csr_matrix(S)
    subs, ncore = [], []
    for C in cores:
        nb = np.unique(np.concatenate([S.indices[S.indptr[i]:S.indptr[i + 1]] for i in C]))
        halo = np.setdiff1d(nb, C, assume_unique=True)
        subs.append(np.concatenate([C, halo]).astype(np.int64))
        ncore.append(len(C))
    return subs, np.array(ncore, dtype=np.int64)


def single_vertex_cores(N):
    """One core per vertex: the subgraphs s_tau^i of Eq. 6 in its original form (Sec. II.A)."""
    return [np.array([i]) for i in range(N)]
