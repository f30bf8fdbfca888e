"""Tight-binding Hamiltonian of the synthetic workloads (oracle side).

The paper builds H with SCC-DFTB in LATTE (Sec. II.B); that code and its parameters are
not available, so the workloads use a one-orbital-per-site model:
  H_ii = onsite_i,
  H_ij = -1.0 * exp(-(r_ij - a) / (0.3 a))  for 0 < r_ij < 2.5 a  (minimum image),
  H_ij = 0 otherwise.
Brute force over all pairs, chunked; obviously correct, O(N^2).
"""
import numpy as np
import scipy.sparse as sp

RCUT = 2.5      # in units of a
DECAY = 0.3     # in units of a


def pair_geometry(pos_i, pos_all, box):
    """Minimum-image distances from rows pos_i to all sites (workload model; the paper's
    SCC-DFTB H of Sec. II.B is not reproduced)."""
    d = pos_i[:, None, :] - pos_all[None, :, :]
    d = d - box * np.round(d / box)
    return np.sqrt(np.einsum("ijk,ijk->ij", d, d))


def hopping(r, a=1.0):
    """Hopping element for separation r (no cutoff applied; workload model, module docstring)."""
    return -1.0 * np.exp(-(r - a) / (DECAY * a))


def build_h(pos, box, onsite, a=1.0, rcut=RCUT, rows=None, chunk=1024):
    """Sparse CSR H of the workload model (module docstring; stands in for Sec. II.B's H),
    float64, sorted column indices, diagonal stored.

    rows: optional subset of row indices; then an [len(rows), N] CSR of those rows.
    """
    pos = np.asarray(pos, dtype=np.float64)
    N = pos.shape[0]
    rows = np.arange(N) if rows is None else np.asarray(rows)
    indptr = [0]
    indices = []
    data = []
    for c0 in range(0, len(rows), chunk):
        rr = rows[c0:c0 + chunk]
        r = pair_geometry(pos[rr], pos, box)
        for k, i in enumerate(rr):
            rk = r[k]
            nb = np.nonzero(rk < rcut * a)[0]
            vals = hopping(rk[nb], a)
            vals[nb == i] = onsite[i]
            indices.append(nb)
            data.append(vals)
            indptr.append(indptr[-1] + len(nb))
    H = sp.csr_matrix((np.concatenate(data), np.concatenate(indices), np.array(indptr)),
                      shape=(len(rows), N))
    H.sort_indices()
    return H


def build_h_tree(pos, box, onsite, a=1.0, rcut=RCUT):
    """The same H as build_h (workload model, module docstring) for systems too large for its
    O(N^2) scan.

    Candidate neighbours come from scipy's periodic k-d tree (a library search, queried
    with a radius slightly above the cutoff); every candidate's distance and hopping are
    then evaluated with the same minimum-image formula as build_h and cut at r < rcut a.
    """
    from scipy.spatial import cKDTree
    pos = np.asarray(pos, dtype=np.float64)
    box = np.asarray(box, dtype=np.float64)
    N = pos.shape[0]
    tree = cKDTree(pos, boxsize=box)
    pr = tree.query_pairs(rcut * a * (1.0 + 1e-9), output_type="ndarray")
    i, j = pr[:, 0], pr[:, 1]
    d = pos[i] - pos[j]
    d = d - box * np.round(d / box)
    r = np.sqrt(np.einsum("ij,ij->i", d, d))
    keep = r < rcut * a
    i, j, v = i[keep], j[keep], hopping(r[keep], a)
    rows = np.concatenate([i, j, np.arange(N)])
    cols = np.concatenate([j, i, np.arange(N)])
    vals = np.concatenate([v, v, np.asarray(onsite, dtype=np.float64)])
    H = sp.csr_matrix((vals, (rows, cols)), shape=(N, N))
    H.sort_indices()
    return H
