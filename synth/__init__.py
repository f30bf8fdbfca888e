"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds random draws and lattice coordinates only: site positions,
species labels, onsite energies drawn per species, and molecular-dynamics
velocities.  It contains none of the method's arithmetic (no Hamiltonian
matrix elements, graph, partition, SP2 or assembly): both the CPU oracle and
the CUDA path build everything else from these arrays on their own.

Workload shapes (the paper's own systems are not available, these stand in):
  * lattice(L): L^3 periodic simple-cubic lattice, one orbital per site at (i+1/2, j+1/2, k+1/2) a,
    rock-salt onsite pattern +1 eV on sites with i+j+k even, -1 eV otherwise,
    positions jittered by N(0, 0.05 a).
  * disordered(N): N sites uniform in a periodic cube at density 1/a^3,
    species 50/50, onsite energies N(+1, 0.1) or N(-1, 0.1) eV by species.
  * velocities(N): per-step displacements N(0, 0.01 a) for the QMD-like run.
"""
import numpy as np


def lattice(L, a=1.0, jitter=0.05, seed=0):
    """L^3 simple-cubic lattice; returns dict(pos[N,3] f64 in [0,box), onsite[N], box[3], grid)."""
    rng = np.random.default_rng(seed)
    g = np.arange(L)
    ijk = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    box = np.full(3, L * a, dtype=np.float64)
    # sites sit at cell centres (i + 1/2) a so that spatial cells of whole lattice
    # spacings hold whole blocks of sites despite the jitter
    pos = (ijk.astype(np.float64) + 0.5) * a + rng.normal(0.0, jitter * a, size=ijk.shape)
    pos = np.mod(pos, box)
    pos[pos >= box] -= box[0]          # np.mod can return box itself for tiny negatives
    onsite = np.where(ijk.sum(axis=1) % 2 == 0, 1.0, -1.0)
    return dict(pos=np.ascontiguousarray(pos), onsite=onsite.astype(np.float64), box=box,
                a=float(a), kind="lattice", L=int(L))


def disordered(N, density=1.0, a=1.0, seed=0, onsite_mean=1.0, onsite_sigma=0.1):
    """N uniform random sites in a periodic cube at the given density (sites per a^3)."""
    rng = np.random.default_rng(seed)
    side = (N / density) ** (1.0 / 3.0) * a
    box = np.full(3, side, dtype=np.float64)
    pos = rng.uniform(0.0, side, size=(N, 3))
    species = rng.integers(0, 2, size=N)
    onsite = np.where(species == 0, onsite_mean, -onsite_mean) + rng.normal(0.0, onsite_sigma, size=N)
    return dict(pos=np.ascontiguousarray(pos), onsite=onsite.astype(np.float64), box=box,
                a=float(a), kind="disordered", species=species.astype(np.int32))


def velocities(N, sigma=0.01, a=1.0, seed=1):
    """Per-step displacement vectors N(0, sigma*a), shape [N,3]."""
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, sigma * a, size=(N, 3))


def advance(pos, vel, box, steps=1):
    """Positions after `steps` constant-velocity steps, wrapped into [0, box).

    The value is np.mod(pos + steps * vel, box), with a result that rounds up to its axis's
    box length moved back by that length.  In a cubic box, when every coordinate stays within one box
    length of [0, box), the wrap is taken with masked in-place adds instead of np.mod (its
    per-element floor and remainder are far slower, and a (3,)-shaped divisor broadcasts in
    inner loops of three): y in [0, b) is unchanged, y in [b, 2b) becomes y - b (exact), and
    y in (-b, 0) becomes fl(y + b), which are np.mod's results on those ranges."""
    y = pos + steps * vel
    b = float(box[0])
    if box[0] == box[1] == box[2] and y.min() > -b and y.max() < 2.0 * b:
        np.add(y, b, out=y, where=y < 0.0)
        np.subtract(y, b, out=y, where=y >= b)
        if y.max() >= b:
            y[y >= b] -= b
        return np.ascontiguousarray(y)
    p = np.mod(y, box)
    p -= box * (p >= box)
    return np.ascontiguousarray(p)
