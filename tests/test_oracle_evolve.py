"""Pins for the oracle's time evolution and observables.

Pinned against: the closed-form one-qubit propagator, second-order convergence
of the Strang split, conservation laws, special schedules that reduce to
trivial evolutions, the adiabatic limit of Sec. 2.1 (the final state approaches
the ground state of H_P as T grows), dense-matrix expectation values, and the
exact factorisation of product instances.
"""

import numpy as np
import pytest

import oracle
import satgen
from oracle.evolve import popcounts


def rabi_closed_form(s, t, psi0):
    """exp(-i t H) psi0 for one qubit, H = (1-s)(1-X)/2 + s |0><0| (clause "x1").

    With a = 1-s, b = s: H = c I + M, c = (a+b)/2, M = (-a X + b Z)/2,
    M^2 = Omega^2 I with Omega = sqrt(a^2 + b^2)/2, hence
    exp(-i t H) = exp(-i c t) [cos(Omega t) I - i sin(Omega t) M / Omega].
    """
    a, b = 1.0 - s, s
    c = 0.5 * (a + b)
    om = 0.5 * np.hypot(a, b)
    X = np.array([[0, 1], [1, 0]], dtype=complex)
    Z = np.diag([1.0, -1.0]).astype(complex)
    M = 0.5 * (-a * X + b * Z)
    U = np.exp(-1j * c * t) * (np.cos(om * t) * np.eye(2) - 1j * np.sin(om * t) * M / om)
    return U @ psi0


PSI0_1Q = np.array([0.6, 0.8j], dtype=complex)


@pytest.mark.parametrize("s", [0.0, 0.25, 0.7, 1.0])
def test_exact_matches_rabi_closed_form(s):
    T, K = 3.7, 5
    got = oracle.evolve_exact(1, [[1]], T, K, psi0=PSI0_1Q, s_values=[s] * K)
    assert np.allclose(got, rabi_closed_form(s, T, PSI0_1Q), atol=1e-12)


def test_strang_converges_to_rabi_at_second_order():
    s, T = 0.4, 5.0
    ref = rabi_closed_form(s, T, PSI0_1Q)
    errs = []
    for K in (20, 40, 80, 160):
        got = oracle.evolve_strang(1, [[1]], T, K, psi0=PSI0_1Q, s_values=[s] * K)
        errs.append(np.max(np.abs(got - ref)))
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(3.7 < r < 4.3 for r in ratios), ratios


def test_strang_vs_exact_second_order_on_sat_instance():
    inst = satgen.planted_instance(5, 1)
    n, cl, T = 5, inst["clauses"], 4.0
    errs = []
    for K in (16, 32, 64):
        ex = oracle.evolve_exact(n, cl, T, K)
        st = oracle.evolve_strang(n, cl, T, K)
        errs.append(np.max(np.abs(ex - st)))
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5, errs


def test_norm_is_conserved():
    inst = satgen.planted_instance(10, 2)
    psi = oracle.evolve_strang(10, inst["clauses"], 8.0, 160)
    assert abs(oracle.norm(psi) - 1.0) < 1e-13


@pytest.mark.parametrize("n", [1, 4, 7])
def test_s_zero_keeps_uniform_state(n):
    cl = satgen.random_instance(n, 3 * n, seed=n, width=min(3, n))
    K = 25
    for fn in (oracle.evolve_strang, oracle.evolve_exact):
        psi = fn(n, cl, 9.0, K, s_values=[0.0] * K)
        assert np.allclose(psi, oracle.uniform_state(n), atol=1e-12)


def test_s_one_keeps_probabilities():
    n, K = 6, 30
    cl = satgen.random_instance(n, 20, seed=4)
    rng = np.random.default_rng(0)
    psi0 = rng.normal(size=64) + 1j * rng.normal(size=64)
    psi0 /= np.sqrt(oracle.norm(psi0))
    psi = oracle.evolve_strang(n, cl, 5.0, K, psi0=psi0, s_values=[1.0] * K)
    assert np.allclose(np.abs(psi) ** 2, np.abs(psi0) ** 2, atol=1e-14)
    e = oracle.violated_counts(n, cl)
    assert np.allclose(psi, np.exp(-1j * 5.0 * e) * psi0, atol=1e-12)


def test_no_clauses_keeps_uniform_state_under_full_schedule():
    psi = oracle.evolve_strang(8, [], 20.0, 100)
    assert np.allclose(psi, oracle.uniform_state(8), atol=1e-12)


def test_adiabatic_limit():
    # Sec. 2.1: a slow enough sweep ends near the ground state of H_P.
    inst = satgen.planted_instance(8, 0)
    e = oracle.violated_counts(8, inst["clauses"])
    assert int(np.count_nonzero(e == 0)) == 1
    ps = []
    for T in (10.0, 40.0, 160.0):
        psi = oracle.evolve_strang(8, inst["clauses"], T, int(round(T / 0.05)), energies=e)
        ps.append(oracle.success_prob(psi, e))
    assert ps[0] < ps[2] and ps[1] < ps[2]
    assert ps[2] > 0.9, ps


def test_merged_half_phases_equal_unmerged():
    # exp(-i a E) exp(-i b E) = exp(-i (a+b) E): merging the half phase of step
    # k with that of step k+1 changes nothing in exact arithmetic.
    n, T, K = 7, 6.0, 40
    inst = satgen.planted_instance(n, 5)
    e = oracle.violated_counts(n, inst["clauses"]).astype(float)
    pc = popcounts(n).astype(float)
    dt = T / K
    s = oracle.midpoint_schedule(K)
    theta = 0.5 * dt * s
    psi = np.exp(-1j * theta[0] * e) * oracle.uniform_state(n)
    for k in range(K):
        psi = oracle.wht_normalized(psi)
        psi = np.exp(-1j * dt * (1 - s[k]) * pc) * psi
        psi = oracle.wht_normalized(psi)
        nxt = theta[k] + (theta[k + 1] if k + 1 < K else 0.0)
        psi = np.exp(-1j * nxt * e) * psi
    ref = oracle.evolve_strang(n, inst["clauses"], T, K)
    assert np.allclose(psi, ref, atol=1e-12)


def test_observables_match_dense_matrices():
    n = 6
    inst = satgen.planted_instance(n, 3)
    cl = inst["clauses"]
    e = oracle.violated_counts(n, cl)
    rng = np.random.default_rng(1)
    psi = rng.normal(size=64) + 1j * rng.normal(size=64)
    psi /= np.sqrt(oracle.norm(psi))
    hb = oracle.hb_dense(n)
    assert abs(oracle.expect_hb(n, psi) - np.vdot(psi, hb @ psi).real) < 1e-12
    for s in (0.0, 0.35, 1.0):
        dense = np.vdot(psi, oracle.h_dense(n, cl, s) @ psi).real
        assert abs(oracle.energy(n, psi, e, s) - dense) < 1e-12
    basis = np.zeros(64, dtype=complex)
    basis[int(np.flatnonzero(e == 0)[0])] = 1.0
    assert oracle.success_prob(basis, e) == 1.0
    assert oracle.expect_hp(basis, e) == 0.0


def test_product_instance_factorises():
    # One-literal clauses only: E(x) = sum_i e_i(x_i), so the Strang state is a
    # tensor product of one-qubit Strang states.
    n, T, K = 5, 7.0, 35
    clauses = [[1], [-2], [3], [3], [-5], [2]]
    e = oracle.violated_counts(n, clauses)
    psi = oracle.evolve_strang(n, clauses, T, K, energies=e)
    factors = []
    for i in range(1, n + 1):
        e0 = sum(1 for c in clauses if c == [i])      # x_i = 0 violates "x_i"
        e1 = sum(1 for c in clauses if c == [-i])     # x_i = 1 violates "NOT x_i"
        factors.append(oracle.one_qubit_strang(e0, e1, T, K))
    for x in range(1 << n):
        amp = 1.0 + 0j
        for i in range(n):
            amp *= factors[i][(x >> i) & 1]
        assert abs(amp - psi[x]) < 1e-12


# ---------------------------------------------------------- fourth order ----
def test_yoshida_weights():
    w1, w0 = oracle.YOSHIDA_W1, oracle.YOSHIDA_W0
    assert abs(2 * w1 + w0 - 1.0) < 1e-15           # consistency
    assert abs(2 * w1 ** 3 + w0 ** 3) < 1e-14       # third-order error cancels
    assert w0 < 0 < w1


def test_substeps_with_equal_lengths_equal_strang():
    inst = satgen.planted_instance(6, 2)
    n, cl, T, K = 6, inst["clauses"], 3.0, 17
    s = oracle.midpoint_schedule(K)
    a = oracle.evolve_substeps(n, cl, np.full(K, T / K), s)
    b = oracle.evolve_strang(n, cl, T, K)
    assert np.max(np.abs(a - b)) < 1e-14


def test_order4_substeps_tile_the_interval():
    T, K = 2.5, 7
    dts, ss = oracle.order4_substeps(T, K)
    assert dts.shape == ss.shape == (3 * K,)
    assert abs(dts.sum() - T) < 1e-13
    # every sub-step's s is the midpoint of its own time interval
    t = np.concatenate([[0.0], np.cumsum(dts)])
    assert np.allclose(ss, 0.5 * (t[:-1] + t[1:]) / T, atol=1e-15)


def test_order4_converges_at_fourth_order_frozen_rabi():
    s, T = 0.4, 5.0
    ref = rabi_closed_form(s, T, PSI0_1Q)
    errs = []
    for K in (10, 20, 40):
        dts, _ = oracle.order4_substeps(T, K)
        got = oracle.evolve_substeps(1, [[1]], dts, np.full(3 * K, s), psi0=PSI0_1Q)
        errs.append(np.max(np.abs(got - ref)))
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    assert all(14.0 < r < 18.0 for r in ratios), ratios


def test_order4_converges_at_fourth_order_time_dependent_sat():
    # linear schedule (H depends on t): reference = fourth order at 8x the steps
    inst = satgen.planted_instance(6, 3)
    n, cl, T = 6, inst["clauses"], 4.0
    ref = oracle.evolve_order4(n, cl, T, 320)
    errs = [np.max(np.abs(oracle.evolve_order4(n, cl, T, K) - ref)) for K in (20, 40)]
    assert 13.0 < errs[0] / errs[1] < 19.0, errs
    # and it beats Strang at equal work (3 Strang sub-steps per fourth-order step)
    strang = np.max(np.abs(oracle.evolve_strang(n, cl, T, 120) - ref))
    assert errs[1] < strang


def _time_ordered_reference(n, clauses, T, psi0):
    """The Schroedinger equation i dpsi/dt = H(t/T) psi of Eq. (1) integrated
    directly (scipy's DOP853 at 1e-12 tolerances): the time-ordered propagator,
    independent of any step schedule."""
    import scipy.integrate
    from oracle.hamiltonian import h_dense
    hb = h_dense(n, clauses, 0.0)
    hp = h_dense(n, clauses, 1.0)

    def rhs(t, y):
        s = t / T
        return -1j * (((1.0 - s) * hb + s * hp) @ y)

    sol = scipy.integrate.solve_ivp(rhs, (0.0, T), psi0.astype(complex), method="DOP853", rtol=1e-12, atol=1e-13)
    assert sol.success
    return sol.y[:, -1]


def test_midpoint_schedule_is_second_order_in_time():
    """Stepping with H frozen at the step midpoints s_k = (k + 1/2)/K converges
    to the time-ordered solution at second order (error ratio 4 when dt halves);
    freezing H at the left end of each step, s = k/K, is only first order
    (ratio 2), so a schedule off by half a step fails here."""
    inst = satgen.planted_instance(3, 2)
    n, cl, T = 3, inst["clauses"], 3.0
    psi0 = oracle.uniform_state(n)
    ref = _time_ordered_reference(n, cl, T, psi0)
    mid, left = [], []
    for K in (10, 20, 40, 80):
        mid.append(np.max(np.abs(oracle.evolve_exact(n, cl, T, K) - ref)))
        left.append(np.max(np.abs(oracle.evolve_exact(n, cl, T, K, s_values=np.arange(K) / K) - ref)))
    r_mid = [mid[i] / mid[i + 1] for i in range(3)]
    r_left = [left[i] / left[i + 1] for i in range(3)]
    assert all(3.6 < r < 4.4 for r in r_mid), r_mid
    assert all(1.7 < r < 2.3 for r in r_left), r_left
    # the Strang split with the same schedule is second order to the same solution
    st = [np.max(np.abs(oracle.evolve_strang(n, cl, T, K) - ref)) for K in (20, 40, 80)]
    assert all(3.5 < st[i] / st[i + 1] < 4.5 for i in range(2)), st


def test_block_instance_factorises():
    """A block instance (clauses never mix blocks) evolves as the tensor product
    of its blocks' Strang states, with the ground-state probability the product
    of theirs: the full-size GPU checks at 30 and 32 qubits rest on this."""
    d = satgen.block_instance(12, 3, 12, 6, seed=9)
    T, K = 2.0, 16
    full = oracle.evolve_strang(12, d["clauses"], T, K)
    x = np.arange(1 << 12)
    prod = np.ones(1 << 12, dtype=complex)
    p_blocks = 1.0
    for blk in d["blocks"]:
        nb = len(blk["vars"])
        e = oracle.violated_counts(nb, blk["clauses"])
        psi = oracle.evolve_strang(nb, blk["clauses"], T, K, energies=e)
        loc = np.zeros(1 << 12, dtype=np.int64)
        for k, v in enumerate(blk["vars"]):
            loc |= ((x >> (v - 1)) & 1) << k
        prod *= psi[loc]
        p_blocks *= oracle.success_prob(psi, e)
    assert np.max(np.abs(full - prod)) <= 1e-12
    e_full = oracle.violated_counts(12, d["clauses"])
    assert abs(oracle.success_prob(full, e_full) - p_blocks) <= 1e-12
