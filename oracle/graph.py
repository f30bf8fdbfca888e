"""Data-dependency graphs S_tau (oracle side).

A graph is returned as a boolean scipy CSR adjacency matrix with sorted column indices,
symmetric, with every diagonal entry present (a vertex always depends on itself).

Readings of the paper used here:
  * Eq. (2) prints {T^(n)(X)}_ij >= tau with no absolute value while the text speaks of
    magnitudes; edges are included when |value| >= tau.
  * A thresholded density matrix is not symmetric (observation i of Sec. II.A); its
    pattern is symmetrised (edge if either |D_ij| or |D_ji| passes) so that the
    core+halo construction sees an undirected graph.
"""
import numpy as np
import scipy.sparse as sp


def _finish(A):
    """Symmetrise, add the diagonal, drop explicit zeros; boolean CSR with sorted indices
    (a graph S_tau has a vertex per row, Sec. II.A; the symmetrised pattern and the
    diagonal are readings of Eq. 2)."""
    A = sp.csr_matrix(A, dtype=bool)
    A = (A + A.T + sp.identity(A.shape[0], dtype=bool, format="csr")).tocsr()
    A.eliminate_zeros()
    A.sort_indices()
    return A.astype(bool)


def pattern(M):
    """Boolean pattern of the stored entries of a sparse matrix (zeros included; helper of the
    Eq. 2 / Eq. 8 graphs)."""
    M = sp.csr_matrix(M)
    P = sp.csr_matrix((np.ones(M.nnz, dtype=bool), M.indices.copy(), M.indptr.copy()), shape=M.shape)
    return P


def h2_threshold(H, thresh):
    """Eq. (2) applied to the square of H: edge (i,j) if |(H^2)_ij| >= thresh."""
    H = sp.csr_matrix(H, dtype=np.float64)
    H2 = (H @ H).tocsr()
    keep = np.abs(H2.data) >= thresh
    A = sp.csr_matrix((keep, H2.indices, H2.indptr), shape=H2.shape)
    return _finish(A)


def d_threshold(D, tau):
    """Pattern of the thresholded density matrix floor(D)_tau: edge if |D_ij| >= tau (Eq. 2 on
    a prior D, as Sec. II.A estimates S_tau from an approximate prior density matrix)."""
    D = sp.csr_matrix(D, dtype=np.float64)
    keep = np.abs(D.data) >= tau
    A = sp.csr_matrix((keep, D.indices, D.indptr), shape=D.shape)
    return _finish(A)


def eq8_symbolic(D, H, tau):
    """Symbolic form of Eq. (8): pattern(floor(D)_tau) union pattern(H), then paths of length <= 2.

    The paper's MD run uses tau = 1e-4 on the previous step's D and epsilon = 0, replacing
    the matrix square by paths of length two in the combined pattern.
    """
    A = (d_threshold(D, tau).astype(np.int64) + pattern(H).astype(np.int64)).tocsr()
    A.data[:] = 1
    A = _finish(A).astype(np.int64)
    A2 = (A @ A).tocsr()
    return _finish(pattern(A2))


def hk_pattern(H, k):
    """Pattern of H^k: vertices joined by a path of length <= k in the pattern of H (a graph
    with extra edges, which obs. iii and viii allow without loss of accuracy)."""
    P = _finish(pattern(H)).astype(np.int64)
    R = P.copy()
    for _ in range(k - 1):
        R = (R @ P).tocsr()
        R = pattern(R).astype(np.int64)
    return _finish(pattern(R))


def complete_blocks(labels):
    """Graph whose connected components are cliques given by equal labels (test helper)."""
    labels = np.asarray(labels)
    N = len(labels)
    rows, cols = [], []
    for lab in np.unique(labels):
        idx = np.nonzero(labels == lab)[0]
        r, c = np.meshgrid(idx, idx, indexing="ij")
        rows.append(r.ravel()); cols.append(c.ravel())
    A = sp.csr_matrix((np.ones(sum(len(r) for r in rows), dtype=bool),
                       (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))
    return _finish(A)


def h2_threshold_rows(H, thresh, rows):
    """Rows `rows` of h2_threshold(H, thresh) (Eq. 2 on H^2), computed from those rows of H^2 alone
    (H^2 is symmetric, so the symmetrisation adds nothing beyond rounding ties); returns
    an N x N boolean CSR whose other rows are empty."""
    H = sp.csr_matrix(H, dtype=np.float64)
    rows = np.asarray(rows)
    R = (H[rows] @ H).tocsr()
    R = sp.csr_matrix((np.abs(R.data) >= thresh, R.indices, R.indptr), shape=R.shape)
    R.eliminate_zeros()
    E = sp.csr_matrix((np.ones(len(rows), dtype=bool), (rows, np.arange(len(rows)))), shape=(H.shape[0], len(rows)))
    A = (E.astype(np.int64) @ R.astype(np.int64)).tocsr()
    A = A + sp.csr_matrix((np.ones(len(rows), dtype=np.int64), (rows, rows)), shape=H.shape)
    A = sp.csr_matrix(A, dtype=bool)
    A.sort_indices()
    return A
