"""Time evolution under Eq. (1) and the observables (test infrastructure only).

Sec. 2.1: the state starts in the ground state of H_B, the uniform superposition
2^(-n/2) sum_x |x>, and evolves by the Schroedinger equation (hbar = 1) while s
sweeps [0, 1] with s = t/T (Eq. (1)).  The paper does not name its integrator;
the readings used here are:

* K equal steps, dt = T/K, and within step k the Hamiltonian is frozen at the
  step midpoint s_k = (k + 1/2)/K  (``midpoint_schedule``).
* ``evolve_exact``: psi <- exp(-i dt H(s_k)) psi with dense exponentials
  (eigendecomposition), the exponential midpoint rule.  Second order in dt.
* ``evolve_strang``: the second-order Strang split of the same step,
      exp(-i dt/2 s_k H_P) . W . exp(-i dt (1-s_k) D) . W . exp(-i dt/2 s_k H_P)
  where W is the normalised Walsh-Hadamard transform and D = diag(popcount),
  because H_B = W D W (the Hadamard maps (I - X)/2 to (I - Z)/2 = |1><1|).
  The two half phases of adjacent steps are deliberately NOT merged here.

All arithmetic is complex128.  ``s_values`` may override the schedule with any
per-step list of s (used for frozen-s closed-form checks).
"""

import numpy as np
import scipy.linalg

from .sat import violated_counts
from .hamiltonian import h_dense


def midpoint_schedule(steps):
    """s_k = (k + 1/2) / K for k = 0 .. K-1 (so s_k = t_mid / T)."""
    k = np.arange(steps, dtype=np.float64)
    return (k + 0.5) / steps


def uniform_state(n):
    """2^(-n/2) on every basis state: the ground state of H_B (Sec. 2.1)."""
    return np.full(1 << n, 2.0 ** (-n / 2.0), dtype=np.complex128)


def popcounts(n):
    x = np.arange(1 << n, dtype=np.int64)
    pc = np.zeros(1 << n, dtype=np.int64)
    for b in range(n):
        pc += (x >> b) & 1
    return pc


def wht_normalized(v):
    """Normalised Walsh-Hadamard transform H^{(x) n} v, one qubit at a time.

    For bit b every pair (x, x + 2^b) with bit b of x clear is replaced by
    (u + w, u - w); the result is scaled once by 2^(-n/2) at the end (exact for
    even n), rather than by a rounded 1/sqrt2 per stage, whose square is not
    exactly 1/2 and would make the norm drift systematically.
    """
    v = np.asarray(v, dtype=np.complex128).copy()
    dim = v.shape[0]
    n = dim.bit_length() - 1
    if 1 << n != dim:
        raise ValueError("length must be a power of two")
    for b in range(n):
        view = v.reshape(dim >> (b + 1), 2, 1 << b)
        u = view[:, 0, :].copy()
        w = view[:, 1, :].copy()
        view[:, 0, :] = u + w
        view[:, 1, :] = u - w
    return v * 2.0 ** (-n / 2.0)


def _schedule(steps, s_values):
    if s_values is None:
        return midpoint_schedule(steps)
    s = np.asarray(s_values, dtype=np.float64)
    if s.shape != (steps,):
        raise ValueError("s_values must have one entry per step")
    return s


def evolve_exact(n, clauses, T, steps, psi0=None, s_values=None):
    """Exponential midpoint rule with dense H(s_k); n <= 10 keeps it quick."""
    dt = T / steps
    psi = uniform_state(n) if psi0 is None else np.asarray(psi0, dtype=np.complex128).copy()
    for s in _schedule(steps, s_values):
        lam, vec = scipy.linalg.eigh(h_dense(n, clauses, s))
        psi = vec @ (np.exp(-1j * dt * lam) * (vec.conj().T @ psi))
    return psi


def evolve_strang(n, clauses, T, steps, psi0=None, s_values=None, energies=None):
    """Second-order Strang split, unmerged half phases, complex128."""
    dt = T / steps
    e = violated_counts(n, clauses) if energies is None else np.asarray(energies)
    e = e.astype(np.float64)
    pc = popcounts(n).astype(np.float64)
    psi = uniform_state(n) if psi0 is None else np.asarray(psi0, dtype=np.complex128).copy()
    for s in _schedule(steps, s_values):
        half_p = np.exp(-1j * (0.5 * dt * s) * e)
        psi = half_p * psi
        psi = wht_normalized(psi)
        psi = np.exp(-1j * (dt * (1.0 - s)) * pc) * psi
        psi = wht_normalized(psi)
        psi = half_p * psi
    return psi


def norm(psi):
    """sum_x |psi_x|^2."""
    psi = np.asarray(psi)
    return float(np.sum(psi.real ** 2 + psi.imag ** 2))


def success_prob(psi, energies):
    """Probability of the ground-state manifold of H_P: sum over E(x) = 0 of |psi_x|^2.

    Sec. 2.1 allows a degenerate final ground state (degeneracy m); summing over
    every zero-energy assignment covers unique and non-unique instances alike.
    """
    psi = np.asarray(psi)
    sel = np.asarray(energies) == 0
    return float(np.sum(np.abs(psi[sel]) ** 2))


def expect_hp(psi, energies):
    """<H_P> = sum_x E(x) |psi_x|^2."""
    return float(np.sum(np.asarray(energies) * np.abs(np.asarray(psi)) ** 2))


def expect_hb(n, psi):
    """<H_B> = n/2 - 1/2 sum_i Re sum_x conj(psi_x) psi_(x XOR 2^(i-1)) (H_B's definition)."""
    psi = np.asarray(psi, dtype=np.complex128)
    x = np.arange(1 << n, dtype=np.int64)
    acc = 0.0
    for i in range(1, n + 1):
        acc += float(np.real(np.vdot(psi, psi[x ^ (1 << (i - 1))])))
    return 0.5 * n * norm(psi) - 0.5 * acc


def energy(n, psi, energies, s):
    """<H(s)> = (1-s) <H_B> + s <H_P>, Eq. (1)."""
    return (1.0 - s) * expect_hb(n, psi) + s * expect_hp(psi, energies)


def evolve_substeps(n, clauses, dt_values, s_values, psi0=None, energies=None):
    """Strang sub-steps of individual lengths dt_j (negative allowed) with H
    frozen at s_j during sub-step j -- the factorisation of ``evolve_strang``
    with a per-sub-step length.  Half phases are not merged."""
    dts = np.asarray(dt_values, dtype=np.float64)
    ss = np.asarray(s_values, dtype=np.float64)
    if dts.shape != ss.shape or dts.ndim != 1:
        raise ValueError("dt_values and s_values must be equal-length vectors")
    e = violated_counts(n, clauses) if energies is None else np.asarray(energies)
    e = e.astype(np.float64)
    pc = popcounts(n).astype(np.float64)
    psi = uniform_state(n) if psi0 is None else np.asarray(psi0, dtype=np.complex128).copy()
    for dt, sv in zip(dts, ss):
        half_p = np.exp(-1j * (0.5 * dt * sv) * e)
        psi = half_p * psi
        psi = wht_normalized(psi)
        psi = np.exp(-1j * (dt * (1.0 - sv)) * pc) * psi
        psi = wht_normalized(psi)
        psi = half_p * psi
    return psi


# Fourth-order triple jump (H. Yoshida, Phys. Lett. A 150, 262 (1990)): a
# symmetric second-order step S(h) composed as S(w1 h) S(w0 h) S(w1 h) with
# 2 w1 + w0 = 1 and 2 w1^3 + w0^3 = 0 is fourth order.  With time carried as an
# extra coordinate, a Strang sub-step that freezes H at the sub-step's midpoint
# time is symmetric, so the composition stays fourth order for H(s(t)).
YOSHIDA_W1 = 1.0 / (2.0 - 2.0 ** (1.0 / 3.0))
YOSHIDA_W0 = 1.0 - 2.0 * YOSHIDA_W1


def order4_substeps(T, steps):
    """(dt_j, s_j) of the 3K sub-steps: step k (dt = T/K, starting at t = k dt)
    is sub-steps of length w1 dt, w0 dt (backwards in time), w1 dt, each with s
    at its own midpoint time divided by T (linear schedule s = t/T)."""
    dt = T / steps
    w = (YOSHIDA_W1, YOSHIDA_W0, YOSHIDA_W1)
    dts, ss = [], []
    for k in range(steps):
        t = k * dt
        for wi in w:
            dts.append(wi * dt)
            ss.append((t + 0.5 * wi * dt) / T)
            t += wi * dt
    return np.asarray(dts), np.asarray(ss)


def evolve_order4(n, clauses, T, steps, psi0=None, energies=None):
    """K fourth-order steps of the linear schedule (3K Strang sub-steps)."""
    dts, ss = order4_substeps(T, steps)
    return evolve_substeps(n, clauses, dts, ss, psi0=psi0, energies=energies)


def one_qubit_strang(e0, e1, T, steps, q0=None, s_values=None):
    """Strang evolution of ONE qubit with H(s) = (1-s)(1 - X)/2 + s diag(e0, e1).

    An instance made only of one-literal clauses has E(x) = sum_i e_i(x_i), and
    both H_B and every Strang factor then factor over qubits, so the n-qubit
    Strang state is the tensor product of these one-qubit states (exactly, in
    real arithmetic).  This gives per-amplitude checks at any n.
    """
    psi = np.array([2 ** -0.5, 2 ** -0.5], dtype=np.complex128) if q0 is None else np.asarray(q0, dtype=np.complex128).copy()
    return evolve_strang(1, [], T, steps, psi0=psi, s_values=s_values,
                         energies=np.array([e0, e1], dtype=np.float64))
