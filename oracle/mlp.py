"""Reference edge classifier that proposes the data-dependency graph (oracle side).

Not in the paper: the graph S_tau of Eq. (2) is normally estimated from a prior density
matrix (Sec. II.A/II.C).  When none exists, a small network scores candidate pairs from
local Hamiltonian features and the pairs it keeps, together with the pattern of H, form
the graph.  This module is the plain FP64 statement of that network:

  candidates  all pairs i != j with minimum-image distance r_ij < rcand
  features    f = [ -log10(max(|H_ij|, 1e-12)) / 12,
                    -log10(max(|(H^2)_ij|, 1e-12)) / 12,
                    r_ij / rcand,
                    min(e_i, e_j), max(e_i, e_j) ]          (e = onsite energies; symmetric in i, j)
  network     h1 = relu(W1 f + b1), h2 = relu(W2 h1 + b2), z = w3 . h2 + b3   (width 64)
              weights used in the forward pass are rounded to fp16 (the master copy is fp32)
  loss        mean binary cross-entropy with logits, label y = 1 when |D_ij| >= tau
  optimiser   Adam (bias-corrected), applied to the fp32 master parameters with the
              gradient taken at the fp16-rounded weights
  graph       pairs with logit >= cut, united with the pattern of H, symmetrised, plus the
              diagonal

Parameter vector layout (4609 for width 64): W1 [64x5] row-major, b1 [64], W2 [64x64]
row-major (out x in), b2 [64], w3 [64], b3 [1].
"""
import numpy as np
import scipy.sparse as sp

from . import graph

NF = 5
HIDDEN = 64


def n_params(h=HIDDEN):
    """Length of the flat parameter vector (layout in the module docstring; not in the paper)."""
    return h * NF + h + h * h + h + h + 1


def unpack(p, h=HIDDEN):
    """Views (W1, b1, W2, b2, w3, b3) of the flat parameter vector (layout in the module docstring)."""
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + h * NF].reshape(h, NF); o += h * NF
    b1 = p[o:o + h]; o += h
    W2 = p[o:o + h * h].reshape(h, h); o += h * h
    b2 = p[o:o + h]; o += h
    w3 = p[o:o + h]; o += h
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def init_params(seed, h=HIDDEN):
    """Seeded He-style initialisation (fp32 values; the learned proposal is not in the paper)."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, np.sqrt(2.0 / NF), (h, NF))
    W2 = rng.normal(0, np.sqrt(2.0 / h), (h, h))
    w3 = rng.normal(0, np.sqrt(1.0 / h), h)
    p = np.concatenate([W1.ravel(), np.zeros(h), W2.ravel(), np.zeros(h), w3, [0.0]])
    return p.astype(np.float32)


def fp16_round(p):
    """Parameters rounded to IEEE half precision (the weights the forward pass uses; module docstring)."""
    return np.asarray(p, dtype=np.float32).astype(np.float16).astype(np.float64)


def candidate_pairs(pos, box, rcand, rows=None):
    """Candidate edges of the learned graph (module docstring; not in the paper): all ordered
    pairs (i, j), i != j, with minimum-image distance < rcand; sorted by (i, j).

    rows: optional ascending subset of i (all rows by default)."""
    N = len(pos)
    I, J, R = [], [], []
    for i in (range(N) if rows is None else rows):
        d = pos[i][None, :] - pos
        d = d - box * np.round(d / box)
        r = np.sqrt(np.einsum("ij,ij->i", d, d))
        js = np.nonzero((r < rcand) & (np.arange(N) != i))[0]
        I.append(np.full(len(js), i)); J.append(js); R.append(r[js])
    return np.concatenate(I), np.concatenate(J), np.concatenate(R)


def features(H, onsite, I, J, R, rcand):
    """Feature matrix [npairs, 5] (FP64) of the module docstring.

    (H^2)_ij = sum_k H_ik H_kj is taken as the dot product of rows i and j (H is
    symmetric), so H may hold only the rows of the sites the pairs touch."""
    H = sp.csr_matrix(H)
    hij = np.asarray(H[I, J]).ravel()
    h2ij = np.asarray(H[I].multiply(H[J]).sum(axis=1)).ravel()
    f = np.empty((len(I), NF))
    f[:, 0] = -np.log10(np.maximum(np.abs(hij), 1e-12)) / 12.0
    f[:, 1] = -np.log10(np.maximum(np.abs(h2ij), 1e-12)) / 12.0
    f[:, 2] = R / rcand
    f[:, 3] = np.minimum(onsite[I], onsite[J])
    f[:, 4] = np.maximum(onsite[I], onsite[J])
    return f


def forward(p, F, h=HIDDEN, cache=False, rounded=True):
    """Logits z of the width-h network for the feature rows F (module docstring)."""
    W1, b1, W2, b2, w3, b3 = unpack(fp16_round(p) if rounded else p, h)
    a1 = F @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    z = h2 @ w3 + b3
    return (z, (h1, h2)) if cache else z


def bce_loss(z, y):
    """Mean binary cross-entropy with logits, numerically stable form (module docstring)."""
    return float(np.mean(np.maximum(z, 0.0) - y * z + np.log1p(np.exp(-np.abs(z)))))


def loss_and_grad(p, F, y, h=HIDDEN, rounded=True):
    """Loss and analytic gradient (back-propagation written out) w.r.t. the (fp16-rounded)
    parameters, FP64; module docstring."""
    W1, b1, W2, b2, w3, b3 = unpack(fp16_round(p) if rounded else p, h)
    z, (h1, h2) = forward(p, F, h, cache=True, rounded=rounded)
    n = len(y)
    dz = (1.0 / (1.0 + np.exp(-z)) - y) / n
    gw3 = h2.T @ dz
    gb3 = dz.sum()
    dh2 = np.outer(dz, w3) * (h2 > 0)
    gW2 = dh2.T @ h1
    gb2 = dh2.sum(axis=0)
    dh1 = (dh2 @ W2) * (h1 > 0)
    gW1 = dh1.T @ F
    gb1 = dh1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, [gb3]])
    return bce_loss(z, y), g


def adam_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One bias-corrected Adam update (Kingma and Ba's published rule); returns (p, m, v) in FP64."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def labels(D, I, J, tau):
    """y = 1 where |D_ij| >= tau (D dense or sparse): the pattern of floor(D)_tau that Sec. II.A
    estimates S_tau from, as training labels."""
    D = sp.csr_matrix(D)
    return (np.abs(np.asarray(D[I, J]).ravel()) >= tau).astype(np.float64)


def graph_from_logits(H, I, J, z, cut):
    """Proposed S_tau (Sec. II.A graph, learned; module docstring): candidate pairs with logit
    z >= cut, united with the pattern of H, symmetrised, with the diagonal (boolean CSR)."""
    N = H.shape[0]
    keep = np.asarray(z) >= cut
    E = sp.csr_matrix((np.ones(int(keep.sum()), dtype=bool), (I[keep], J[keep])), shape=(N, N))
    return graph._finish(E + graph.pattern(H))
