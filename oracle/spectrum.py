"""Lowest eigenvalues of H(s) (Eq. (1)) by dense diagonalisation (test
infrastructure only; n <= 12).

The adiabatic evolution of Sec. 2.1 stays in the ground state if it is slow
compared with the gap between the two lowest levels that the state can reach.
Starting from the uniform superposition, the reachable levels are those whose
eigenspaces overlap the uniform state (the Krylov space of H(s) from it):
``sector_eigenvalues`` keeps exactly those, grouping numerically equal
eigenvalues into one level and summing the overlap over its eigenspace.
"""

import numpy as np
import scipy.linalg

from .hamiltonian import h_dense


def eigenvalues(n, clauses, s):
    """All eigenvalues of the dense H(s), ascending."""
    return scipy.linalg.eigvalsh(h_dense(n, clauses, s))


def sector_eigenvalues(n, clauses, s, k, weight_tol=1e-10, level_tol=1e-9):
    """The k lowest distinct levels of H(s) whose eigenspace overlaps the
    uniform state (total squared overlap > weight_tol), ascending."""
    lam, vec = scipy.linalg.eigh(h_dense(n, clauses, s))
    u = np.full(1 << n, 2.0 ** (-n / 2.0))
    w = np.abs(vec.conj().T @ u) ** 2
    levels = []
    i = 0
    while i < len(lam) and len(levels) < k:
        j = i
        while j + 1 < len(lam) and lam[j + 1] - lam[i] <= level_tol:
            j += 1
        if w[i:j + 1].sum() > weight_tol:
            levels.append(float(np.mean(lam[i:j + 1])))
        i = j + 1
    return np.array(levels)


def sector_gap(n, clauses, s):
    """E1 - E0 of the levels reachable from the uniform state (nan if fewer than two)."""
    lv = sector_eigenvalues(n, clauses, s, 2)
    return float(lv[1] - lv[0]) if len(lv) >= 2 else float("nan")


def sparse_levels(n, clauses, s, k, level_tol=1e-8):
    """The k lowest distinct levels of H(s) for larger n, from a sparse H
    (H_B as the n bit-flip terms, H_P diagonal) and ARPACK (scipy eigsh) as the
    eigensolver step; degenerate copies merge within level_tol."""
    import scipy.sparse
    import scipy.sparse.linalg
    from .sat import violated_counts
    dim = 1 << n
    x = np.arange(dim, dtype=np.int64)
    rows, cols, vals = [x], [x], [0.5 * n * (1.0 - s) + s * violated_counts(n, clauses).astype(np.float64)]
    for i in range(n):
        rows.append(x)
        cols.append(x ^ (1 << i))
        vals.append(np.full(dim, -0.5 * (1.0 - s)))
    h = scipy.sparse.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(dim, dim))
    lam = np.sort(scipy.sparse.linalg.eigsh(h, k=min(dim - 2, 4 * k + 8), which="SA", tol=1e-12)[0])
    levels = []
    for v in lam:
        if not levels or v - levels[-1] > level_tol:
            levels.append(float(v))
    return np.array(levels[:k])
