"""K-SAT semantics and the final-Hamiltonian energy, by brute force.

Test infrastructure (see the package docstring): only tests, ``smoke()`` and the
CPU-baseline leg of ``bench.py`` may use it.

Sec. 2.2 defines a K-SAT instance P as a conjunction of clauses, each clause a
disjunction of literals drawn from {e_i, NOT e_i}; P is satisfied when every
clause holds.  Sec. 4.3 builds the final Hamiltonian from an energy function
that gives every assignment an energy proportional to its number of unsatisfied
clauses, a sum of one term per clause.  With the proportionality constant taken
as 1, E(x) is the integer count of clauses that assignment x leaves false.
A clause is false exactly when every one of its literals is false.

Bit convention (Sec. 2.1 basis order |q_n ... q_1>): x_i is bit (i-1) of x.
Repeated clauses are counted with multiplicity (the paper's own worked instance
contains two repeats).
"""

import numpy as np


def _literal_value(x_bits_of_var, lit):
    """Truth value of literal ``lit`` given the 0/1 value(s) of its variable."""
    if lit > 0:
        return x_bits_of_var == 1
    return x_bits_of_var == 0


def clause_is_violated(x, clause):
    """True when assignment ``x`` (a Python int) makes every literal of ``clause`` false."""
    for lit in clause:
        if lit == 0:
            continue
        bit = (int(x) >> (abs(int(lit)) - 1)) & 1
        if _literal_value(bit, lit):
            return False
    return True


def energy_at(n, clauses, x):
    """E(x): number of clauses violated by assignment x (one assignment, pure Python).

    Used for sampled checks at sizes where the full diagonal does not fit.
    """
    if not (0 <= int(x) < (1 << n)):
        raise ValueError("assignment out of range")
    return sum(1 for c in clauses if clause_is_violated(x, c))


def violated_counts(n, clauses):
    """E(x) for every x in [0, 2^n): the diagonal of the final Hamiltonian H_P.

    Vectorised over x but otherwise the definition: for each clause, an
    assignment violates it when all its literals evaluate to false.
    """
    if n > 26:
        raise ValueError("brute-force diagonal is limited to n <= 26")
    x = np.arange(1 << n, dtype=np.int64)
    counts = np.zeros(1 << n, dtype=np.int64)
    for clause in clauses:
        all_false = np.ones(1 << n, dtype=bool)
        for lit in clause:
            lit = int(lit)
            if lit == 0:
                continue
            v = abs(lit)
            if v > n:
                raise ValueError("literal refers to a variable beyond n")
            bits = (x >> (v - 1)) & 1
            all_false &= ~_literal_value(bits, lit)
        counts += all_false
    return counts


def count_solutions(n, clauses):
    """Number of satisfying assignments (E(x) == 0), by enumeration."""
    return int(np.count_nonzero(violated_counts(n, clauses) == 0))
