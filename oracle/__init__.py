"""CPU oracle for graph-partitioned SP2 density matrices (test infrastructure).

Plain, slow, FP64 NumPy/SciPy restatement of what the CUDA path computes, written
from the paper (Niklasson et al., "Graph-based linear scaling electronic structure
theory") and from the published SP2 recursion it cites.  It exists only to check the
CUDA path: the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import it; the product package never does, and nothing here imports the
product package.

Modules
  hamiltonian  tight-binding H from positions (workload model; not in the paper)
  graph        data-dependency graphs S_tau: Eq. (2), Eq. (8), H^k patterns
  partition    cores (communities) and core+halo subgraphs (Sec. II.A, Fig. 1)
  sp2          Gershgorin bounds, dense SP2, thresholded sparse SP2 (Eqs. 3-5),
               graph-partitioned SP2 with column assembly (Eq. 6), serial
               Chebyshev expansion identity (Eqs. 1, 4-6)
  exact        zero-temperature density matrix by diagonalisation
  mlp          reference edge-classifier MLP (forward, BCE, backward, Adam)

Pins (tests/test_oracle_*.py) tie each function to closed forms, textbook routines,
brute force and the paper's exact Eq. (6) identity; see the module docstrings.
tests/test_oracle_mutants.py plants plausible mistakes in these modules' source, one at
a time, and checks that a pin catches each.
"""
