"""Zero-temperature density matrix by exact diagonalisation.

D = theta(mu I - H) = V_occ V_occ^T, the lowest n_occ eigenvectors of H, which is the
limit the paper's recursive expansion converges to (Sec. II.A, zero-temperature limit of
Eq. (7)).  LAPACK eigh; feasible up to a few thousand orbitals.
"""
import numpy as np


def density_matrix(H, n_occ):
    """Zero-temperature D = theta(mu I - H) (Sec. II.A, the zero-temperature limit of Eq. 7):
    the projector on the n_occ lowest eigenvectors, by LAPACK eigh.  Returns (D, eigenvalues)."""
    Hd = H.toarray() if hasattr(H, "toarray") else np.asarray(H)
    w, V = np.linalg.eigh(Hd)
    Vo = V[:, :n_occ]
    return Vo @ Vo.T, w


def homo_lumo(H, n_occ):
    """Highest occupied and lowest unoccupied eigenvalues (the gap that fixes the SP2
    sequence of the MD run, Sec. II.C)."""
    _, w = density_matrix(H, n_occ)
    return w[n_occ - 1], w[n_occ]
