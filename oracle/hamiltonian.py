"""Dense Hamiltonians of Eq. (1) for small n (test infrastructure only).

Eq. (1):  H(s) = (1 - s) H_i + s H_f,  s = t / tau.

* H_i ("beginning" Hamiltonian, written H_B here): Sec. 2.1 only asks that its
  ground state be the uniform superposition of all 2^n basis states.  The
  reading used throughout is the transverse field H_B = sum_i (I - X_i)/2, whose
  unique ground state (energy 0) is that uniform superposition.
* H_f ("problem" Hamiltonian, written H_P here): diag(E(x)) with E the
  violated-clause count of Sec. 4.3 (see ``oracle.sat``).

Matrices are built with ``np.kron`` in the order q_n (x) ... (x) q_1 of Sec. 2.1,
so that the first Kronecker factor is the most significant bit of the index
x = sum_i q_i 2^(i-1).
"""

import numpy as np

from .sat import violated_counts

_X = np.array([[0.0, 1.0], [1.0, 0.0]], dtype=np.complex128)
_I2 = np.eye(2, dtype=np.complex128)


def sigma_x_dense(n, i):
    """X_i acting on qubit q_i (1-based), i.e. on bit (i-1) of the index."""
    if not 1 <= i <= n:
        raise ValueError("qubit index out of range")
    out = np.ones((1, 1), dtype=np.complex128)
    for q in range(n, 0, -1):  # q_n first: most significant factor
        out = np.kron(out, _X if q == i else _I2)
    return out


def hb_dense(n):
    """H_B = sum_i (I - X_i)/2 as a dense 2^n x 2^n matrix."""
    dim = 1 << n
    h = np.zeros((dim, dim), dtype=np.complex128)
    eye = np.eye(dim, dtype=np.complex128)
    for i in range(1, n + 1):
        h += 0.5 * (eye - sigma_x_dense(n, i))
    return h


def hp_dense(n, clauses):
    """H_P = diag(E(x)) as a dense matrix."""
    return np.diag(violated_counts(n, clauses).astype(np.complex128))


def h_dense(n, clauses, s):
    """H(s) = (1-s) H_B + s H_P, Eq. (1)."""
    if n > 12:
        raise ValueError("dense Hamiltonians are limited to n <= 12")
    return (1.0 - s) * hb_dense(n) + s * hp_dense(n, clauses)
