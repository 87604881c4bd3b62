"""Oracle: a plain, slow, obviously correct CPU model of adiabatic 3-SAT evolution.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it.  It shares no code with the CUDA path (no kernels, headers,
tables or helpers); the only module both sides consume is ``satgen`` (seeded
instance generation, which holds none of the evolution arithmetic).

Everything is complex128 / float64 NumPy, written in the order of the paper:

* ``sat``          -- the K-SAT proposition of Sec. 2.2 and the final-Hamiltonian
                      energy of Sec. 4.3 ("energy proportional to the number of
                      unsatisfied clauses", proportionality constant 1): E(x) by
                      brute force over all assignments.
* ``hamiltonian``  -- dense H(s) = (1-s) H_B + s H_P of Eq. (1) for small n, with
                      H_B = sum_i (1 - sigma^x_i)/2 whose ground state is the
                      uniform superposition of Sec. 2.1.
* ``evolve``       -- time evolution: exponential midpoint rule with dense
                      exponentials (small n) and the second-order Strang split
                      (unmerged half phases, explicit Walsh-Hadamard transform),
                      plus the observables (norm, ground-state probability,
                      <H(s)>).

Conventions (Sec. 2.1): basis state |q_n ... q_1>, q_i = 0 is the sigma^z = +1
state; the integer index is x = sum_i q_i 2^(i-1), i.e. variable x_i of the
3-SAT instance is bit i-1 of x.  Clauses are lists of signed 1-based literals
(+i means x_i, -i means NOT x_i); 0 entries are ignored padding.

Parity pins: every function here is pinned by ``tests/test_oracle_*.py`` against
values fixed by the paper or by mathematics (worked example of Sec. 2.2, closed
form one-qubit evolution, spectra, invariants, convergence order).  No function
is "parity unpinned".
"""

from .sat import violated_counts, energy_at, count_solutions, clause_is_violated
from .hamiltonian import hb_dense, hp_dense, h_dense, sigma_x_dense
from .spectrum import eigenvalues, sector_eigenvalues, sector_gap, sparse_levels
from .evolve import (
    midpoint_schedule,
    uniform_state,
    wht_normalized,
    evolve_exact,
    evolve_strang,
    norm,
    success_prob,
    expect_hp,
    expect_hb,
    energy,
    one_qubit_strang,
    evolve_substeps,
    order4_substeps,
    evolve_order4,
    YOSHIDA_W0,
    YOSHIDA_W1,
)

__all__ = [
    "violated_counts", "energy_at", "count_solutions", "clause_is_violated",
    "hb_dense", "hp_dense", "h_dense", "sigma_x_dense",
    "midpoint_schedule", "uniform_state", "wht_normalized", "evolve_exact",
    "evolve_strang", "norm", "success_prob", "expect_hp", "expect_hb", "energy",
    "one_qubit_strang",
]
