"""SP2 recursive Fermi-operator expansion: dense, thresholded sparse, graph-partitioned.

Zero-temperature density matrix D = theta(mu I - H) as the limit of nested 2nd-order
polynomials f_n (Sec. II.A, the SP2 scheme the paper cites and uses in Secs. II.B-C).
The paper names SP2 but does not print its steps; this module states the published
form:
  1. Gershgorin bounds e_min = min_i (H_ii - sum_{j!=i} |H_ij|),
                       e_max = max_i (H_ii + sum_{j!=i} |H_ij|).
  2. X_0 = (e_max I - H) / (e_max - e_min)        (spectrum mapped into [0, 1], reversed)
  3. for n = 0, 1, ...:  t1 = Tr X_n, t2 = Tr X_n^2, e_n = |t1 - t2|;
        stop when e_n <= idem_tol (or a stall / n_max / replay-length rule below);
        X_{n+1} = X_n^2       if |t2 - N_occ| < |2 t1 - t2 - N_occ|   (branch bit 1)
        X_{n+1} = 2X_n - X_n^2 otherwise                              (branch bit 0)
Readings (paper silent): ties go to 2X - X^2; a stall stop fires when n >= n_min and
e_n >= e_{n-2}; "replay" mode applies a given branch sequence and stops after it.

Graph-partitioned form (Eq. 6, observation vi): every core+halo subgraph s takes the
principal submatrix x_s = X_0[idx_s, idx_s] and runs the same branch sequence, the
traces being summed over core positions of all subgraphs (one global expansion); column
C_s[j] of D is column j of the final x_s.  Thresholded sparse form (Eqs. 3-5): every
product is followed by floor(.)_S.
"""
import numpy as np
import scipy.sparse as sp


def gershgorin(H):
    """Gershgorin bounds (e_min, e_max) of the spectrum of the whole H: the spectral scaling
    of the recursive expansion cited in Sec. II.A (every subgraph shares them)."""
    H = sp.csr_matrix(H)
    d = H.diagonal()
    off = np.asarray(abs(H).sum(axis=1)).ravel() - np.abs(d)
    return float(np.min(d - off)), float(np.max(d + off))


def choose_square(t1, t2, n_occ):
    """Branch rule of the SP2 recursion (Sec. II.A, cited): True selects X^2, False 2X - X^2;
    the choice that moves the trace toward n_occ (a tie selects 2X - X^2)."""
    return abs(t2 - n_occ) < abs(2.0 * t1 - t2 - n_occ)


class Log:
    """Per-step record of an SP2 run (Sec. II.A recursion): branch bits, traces t1 = Tr X_n,
    t2 = Tr X_n^2, e_n."""
    def __init__(self):
        self.seq, self.t1, self.t2, self.e = [], [], [], []
        self.stop = None

    @property
    def iters(self):
        return len(self.seq)


def _decide(log, n, t1, t2, n_occ, idem_tol, n_min, n_max, seq):
    """Record traces of X_n and return the branch bit, or None to stop (idempotency tolerance,
    stall rule or n_max in global mode; the given sequence in replay mode, Sec. II.C)."""
    e = abs(t1 - t2)
    log.t1.append(t1); log.t2.append(t2); log.e.append(e)
    if seq is not None:
        if n >= len(seq):
            log.stop = "replay"
            return None
        return bool(seq[n])
    if e <= idem_tol:
        log.stop = "tol"
        return None
    if n >= n_min and n >= 2 and e >= log.e[n - 2]:
        log.stop = "stall"
        return None
    if n >= n_max:
        log.stop = "nmax"
        return None
    return choose_square(t1, t2, n_occ)


def initial_x(H, eps):
    """X_0 = (e_max I - H) / (e_max - e_min): H mapped into [0, 1] with the occupied end at 1
    (the recursive expansion of Sec. II.A starts from this)."""
    e_min, e_max = eps
    H = sp.csr_matrix(H, dtype=np.float64)
    N = H.shape[0]
    return ((e_max * sp.identity(N, format="csr") - H) / (e_max - e_min)).tocsr()


def sp2_dense(H, n_occ, idem_tol=1e-10, n_min=10, n_max=100, seq=None, eps=None):
    """Dense FP64 SP2 on the whole matrix (the recursive expansion of Sec. II.A without any
    threshold).  Returns (D, log)."""
    eps = gershgorin(H) if eps is None else eps
    X = initial_x(H, eps).toarray()
    log = Log()
    n = 0
    while True:
        S = X @ X
        b = _decide(log, n, float(np.trace(X)), float(np.trace(S)), n_occ, idem_tol, n_min, n_max, seq)
        if b is None:
            return X, log
        X = S if b else 2.0 * X - S
        log.seq.append(int(b))
        n += 1


def threshold_to(A, S):
    """floor(A)_S of Eq. (3): keep entries on edges of S, zero elsewhere (sparse result)."""
    A = sp.csr_matrix(A)
    M = A.multiply(sp.csr_matrix(S, dtype=np.float64))
    M = sp.csr_matrix(M)
    M.eliminate_zeros()
    return M


def sp2_thresholded(H, S, n_occ, idem_tol=1e-10, n_min=10, n_max=100, seq=None, eps=None):
    """Globally thresholded sparse SP2 (Eqs. 3-5 with SP2 products).  Returns (X sparse, log)."""
    eps = gershgorin(H) if eps is None else eps
    X = threshold_to(initial_x(H, eps), S)
    log = Log()
    n = 0
    while True:
        Sq = threshold_to(X @ X, S)
        b = _decide(log, n, float(X.diagonal().sum()), float(Sq.diagonal().sum()),
                    n_occ, idem_tol, n_min, n_max, seq)
        if b is None:
            return X, log
        X = Sq if b else (2.0 * X - Sq).tocsr()
        log.seq.append(int(b))
        n += 1


def gather_submatrices(H, subs, eps):
    """x_s = X_0[idx_s, idx_s] for each subgraph: the dense principal submatrices x[s] of Eq. 6
    (dense FP64)."""
    X0 = initial_x(H, eps)
    return [X0[idx][:, idx].toarray() for idx in subs]


def sp2_graph(H, subs, ncore, n_occ, idem_tol=1e-10, n_min=10, n_max=100, seq=None, eps=None,
              return_subs=False):
    """Graph-partitioned SP2 (Eq. 6 with a global SP2 branch sequence).

    subs: local index lists (cores first); ncore: core count per subgraph.
    Returns (D as scipy CSC [N,N], log) where D[:, C_s[j]] = x_s[:, j].
    """
    eps = gershgorin(H) if eps is None else eps
    xs = gather_submatrices(H, subs, eps)
    log = Log()
    n = 0
    while True:
        Ss = [x @ x for x in xs]
        t1 = sum(float(np.trace(x[:c, :c])) for x, c in zip(xs, ncore))
        t2 = sum(float(np.trace(s[:c, :c])) for s, c in zip(Ss, ncore))
        b = _decide(log, n, t1, t2, n_occ, idem_tol, n_min, n_max, seq)
        if b is None:
            break
        xs = [s if b else 2.0 * x - s for x, s in zip(xs, Ss)]
        log.seq.append(int(b))
        n += 1
    D = assemble(xs, subs, ncore, H.shape[0])
    return (D, log, xs) if return_subs else (D, log)


def assemble(xs, subs, ncore, N, drop_tol=0.0):
    """Column assembly of Eq. (6): D[idx_s[k], idx_s[j]] = x_s[k, j] for core positions j.

    Entries with |value| < drop_tol are omitted (drop_tol = 0 keeps everything).
    """
    rows, cols, vals = [], [], []
    for x, idx, c in zip(xs, subs, ncore):
        blk = x[:, :c]
        r = np.repeat(idx[:, None], c, axis=1)
        cc = np.repeat(idx[None, :c], len(idx), axis=0)
        keep = np.abs(blk) >= drop_tol
        rows.append(r[keep]); cols.append(cc[keep]); vals.append(blk[keep])
    return sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))


def chebyshev_thresholded(X, S, coeffs):
    """P_tau(X) = sum_n c_n T^(n)_S(X) with T_0 = I, T_1 = floor(X)_S,
    T_n = 2 floor(X T_{n-1})_S - T_{n-2}  (Eqs. 4-5 with Chebyshev alpha's)."""
    N = X.shape[0]
    T0 = sp.identity(N, format="csr")
    T1 = threshold_to(X, S)
    P = coeffs[0] * T0 + coeffs[1] * T1
    for c in coeffs[2:]:
        T2 = (2.0 * threshold_to(X @ T1, S) - T0).tocsr()
        P = P + c * T2
        T0, T1 = T1, T2
    return sp.csr_matrix(P)


def chebyshev_dense(x, coeffs):
    """Dense P(x) = sum_n c_n T_n(x) (Eq. 1 with Chebyshev T_n), T_0 = I, T_1 = x,
    T_n = 2 x T_{n-1} - T_{n-2}."""
    m = x.shape[0]
    T0 = np.eye(m)
    T1 = x.copy()
    P = coeffs[0] * T0 + coeffs[1] * T1
    for c in coeffs[2:]:
        T2 = 2.0 * x @ T1 - T0
        P = P + c * T2
        T0, T1 = T1, T2
    return P


def chebyshev_graph(X, subs, coeffs):
    """Column i of P from the dense polynomial of the subgraph of single-vertex core i (Eq. 6)."""
    X = sp.csr_matrix(X)
    N = X.shape[0]
    rows, cols, vals = [], [], []
    for idx in subs:
        x = X[idx][:, idx].toarray()
        p = chebyshev_dense(x, coeffs)[:, 0]
        rows.append(idx); cols.append(np.full(len(idx), idx[0])); vals.append(p)
    return sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))


# ---------------------------------------------------------------- pre-determined sequences
# Sec. II.C: in the MD run every step's branch sequence is fixed beforehand from a HOMO-LUMO
# gap estimated at the previous step.  Readings (the cited estimator is not printed):
#  * the estimate models a late SP2 step as two unconverged levels, the HOMO image x_h (near
#    1) and the LUMO image x_l (near 0), every other level being converged:
#        Tr X_k - Tr X_k^2 = x_h (1 - x_h) + x_l (1 - x_l),   Tr X_k - N_occ = (x_h - 1) + x_l,
#    solved for (x_h, x_l) and mapped back through the inverse branch maps to eigenvalues;
#  * the sequence applies the branch rule above to the two-level matrix diag(x_h, x_l) with
#    one occupied level, until both are within tol of 1 and 0.
def gap_estimate(t1, t2, seq, n_occ, eps, e_lo, e_hi):
    """(homo, lumo) from the traces of a finished run (Sec. II.C; reading in the comment
    above); uses the last step whose idempotency error lies in [e_lo, e_hi]."""
    ks = [k for k in range(min(len(t1), len(t2))) if e_lo <= t1[k] - t2[k] <= e_hi]
    if not ks:
        raise ValueError("no step with idempotency error in range")
    k = ks[-1]
    e, d = t1[k] - t2[k], t1[k] - n_occ
    # substitute x_l = d + 1 - x_h into the first equation: a quadratic in x_h
    c = d + 1.0
    roots = np.roots([-2.0, 2.0 * c, c - c * c - e])
    xh = float(max(r.real for r in roots if abs(r.imag) < 1e-12))
    xl = c - xh
    for b in reversed(seq[:k]):
        if b:
            xh, xl = np.sqrt(xh), np.sqrt(xl)
        else:
            xh, xl = 1.0 - np.sqrt(1.0 - xh), 1.0 - np.sqrt(1.0 - xl)
    e_min, e_max = eps
    return e_max - xh * (e_max - e_min), e_max - xl * (e_max - e_min)


def sequence_from_gap(eps, homo, lumo, tol, n_max=256):
    """Branch sequence fixed beforehand from a HOMO-LUMO estimate (Sec. II.C; reading in the
    comment above): the branch rule applied to the two-level model until both levels are
    within tol of 1 and 0."""
    e_min, e_max = eps
    xh = (e_max - homo) / (e_max - e_min)
    xl = (e_max - lumo) / (e_max - e_min)
    seq = []
    while not (1.0 - xh <= tol and xl <= tol):
        if len(seq) == n_max:
            raise RuntimeError("sequence longer than n_max")
        b = choose_square(xh + xl, xh * xh + xl * xl, 1.0)
        xh, xl = (xh * xh, xl * xl) if b else (2 * xh - xh * xh, 2 * xl - xl * xl)
        seq.append(int(b))
    return seq


# ---------------------------------------------------------------- finite temperature (Eq. 7)
# D = [exp(beta (H - mu)) + 1]^-1 ~ sum_n c_n T_n(x), x = (H - a I) / b on the Gershgorin
# interval [e_min, e_max] (a its centre, b its half-width).  Readings: the coefficients are
# the Chebyshev interpolant of the Fermi function at K = 2 (order + 1) Chebyshev-Gauss
# nodes (c_n = (2 - delta_n0) / K sum_j f(a + b cos t_j) cos(n t_j), t_j = pi (j + 1/2) / K);
# the series is evaluated per subgraph with Clenshaw's recurrence
#   b_k = c_k I + 2 x b_{k+1} - b_{k+2} (k = order .. 1, b_{order+1} = b_{order+2} = 0),
#   P = c_0 I + x b_1 - b_2,
# which is the same polynomial as the forward sum of c_n T_n (Eqs. 4-5) in another order.
def fermi(e, beta, mu):
    """Fermi function [exp(beta (e - mu)) + 1]^-1 of Eq. 7, in a form without overflow."""
    z = beta * (np.asarray(e, dtype=np.float64) - mu)
    return 0.5 * (1.0 - np.tanh(0.5 * z))


def fermi_chebyshev_coeffs(beta, mu, eps, order):
    """Chebyshev coefficients c_n of the Fermi function of Eq. 7 on [e_min, e_max]
    (interpolant at Chebyshev-Gauss nodes; reading in the comment above)."""
    e_min, e_max = eps
    a, b = 0.5 * (e_max + e_min), 0.5 * (e_max - e_min)
    K = 2 * (order + 1)
    t = np.pi * (np.arange(K) + 0.5) / K
    f = fermi(a + b * np.cos(t), beta, mu)
    n = np.arange(order + 1)
    c = (2.0 / K) * (np.cos(np.outer(n, t)) @ f)
    c[0] *= 0.5
    return c


def clenshaw_dense(x, coeffs):
    """sum_n c_n T_n(x) for a dense x by Clenshaw's recurrence (the same polynomial as the
    forward sum of Eqs. 1, 4-5, in another order; obs. ix allows any order here)."""
    m = x.shape[0]
    b1 = np.zeros((m, m))
    b2 = np.zeros((m, m))
    for c in coeffs[:0:-1]:          # c_order .. c_1
        b1, b2 = c * np.eye(m) + 2.0 * x @ b1 - b2, b1
    return coeffs[0] * np.eye(m) + x @ b1 - b2


def foe_graph(H, subs, ncore, beta, mu, order, eps=None, coeffs=None, return_subs=False):
    """Graph-partitioned finite-temperature D (Eq. 7 per subgraph, assembled by Eq. 6)."""
    H = sp.csr_matrix(H, dtype=np.float64)
    eps = gershgorin(H) if eps is None else eps
    coeffs = fermi_chebyshev_coeffs(beta, mu, eps, order) if coeffs is None else coeffs
    a, b = 0.5 * (eps[1] + eps[0]), 0.5 * (eps[1] - eps[0])
    xs = []
    for idx in subs:
        h = H[idx][:, idx].toarray()
        xs.append(clenshaw_dense((h - a * np.eye(len(idx))) / b, coeffs))
    D = assemble(xs, subs, ncore, H.shape[0])
    return (D, coeffs, xs) if return_subs else (D, coeffs)
