"""GPU parity: the CUDA path (through the C ABI) against the complex128 oracle.

Bars (stated for the method): E(x) bit exact; max amplitude error <= 1e-5 for the
FP32 path; probabilities within 1e-6.  The ground-state probability is checked
as returned (raw) and as the Born probability of the normalised state,
P / ||psi||^2, both within 1e-6.  Every low pass folds the FP32 state's norm
back to its starting value (the norm fold), so the norm itself stays within
1e-6 (NORM_TOL) instead of drifting by a random walk of roundings.  Sizes span the on-chip evolver (n <= 14),
the two-group streaming plan (n = 15..20, every strided width 5..10) and the
three-group plan (n >= 21), with ragged widths.
"""

import numpy as np
import pytest

import oracle
import satgen

pytestmark = pytest.mark.gpu

AMP_TOL = 1e-5
PROB_TOL = 1e-6
NORM_TOL = 1e-6


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need a CUDA device"
    return t


@pytest.fixture(scope="module")
def q(torch):
    import paper_1103_1399_gb300 as q
    return q


def paper_instance():
    import json
    import os
    from conftest import GOLDEN
    with open(os.path.join(GOLDEN, "paper_instance.json")) as f:
        d = json.load(f)
    return d["n"], d["clauses"]


def gpu_diag(q, torch, n, clauses):
    inst = q.Instance(n, clauses)
    out = torch.empty(1 << n, dtype=torch.int16, device="cuda")
    inst.hp_diagonal(out)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint16).astype(np.int64)


def to_gpu(torch, psi):
    return torch.from_numpy(np.ascontiguousarray(psi, dtype=np.complex64)).cuda()


def to_np(psi):
    return psi.cpu().numpy().astype(np.complex128)


# ---------------------------------------------------------------- E(x) ------
DIAG_CASES = [
    ("paper", None),
    ("n1", (1, [[1]])),
    ("n1-neg-dup", (1, [[-1], [-1], [1]])),
    ("n2-width1", (2, [[1], [-2]])),
    ("n3-empty", (3, [])),
    ("n9-rand", (9, satgen.random_instance(9, 40, seed=1))),
    ("n10-rand", (10, satgen.random_instance(10, 200, seed=2))),
    ("n11-rand", (11, satgen.random_instance(11, 57, seed=3))),
    ("n12-planted", None),
    ("n12-max-m", (12, satgen.random_instance(12, 1023, seed=4))),
    ("n13-mixed-width", (13, satgen.random_instance(13, 30, seed=5, width=1) + satgen.random_instance(13, 30, seed=6, width=2)
                         + satgen.random_instance(13, 60, seed=7))),
    ("n17-rand", (17, satgen.random_instance(17, 120, seed=8))),
    ("n20-planted", None),
    ("n21-rand", (21, satgen.random_instance(21, 160, seed=9))),
]


@pytest.mark.parametrize("name,case", DIAG_CASES, ids=[c[0] for c in DIAG_CASES])
def test_hp_diagonal_bit_exact(q, torch, name, case):
    if name == "paper":
        n, cl = paper_instance()
    elif name == "n12-planted":
        d = satgen.load_instance("planted_n12_s0")
        n, cl = d["n"], d["clauses"]
    elif name == "n20-planted":
        d = satgen.load_instance("planted_n20_s0")
        n, cl = d["n"], d["clauses"]
    else:
        n, cl = case
    got = gpu_diag(q, torch, n, cl)
    ref = oracle.violated_counts(n, cl)
    assert np.array_equal(got, ref)


def test_paper_instance_solution_on_gpu(q, torch):
    n, cl = paper_instance()
    e = gpu_diag(q, torch, n, cl)
    assert np.flatnonzero(e == 0).tolist() == [10]


# ---------------------------------------------------------------- evolve ----
def run_gpu(q, torch, n, cl, T, K, psi0=None):
    inst = q.Instance(n, cl)
    if psi0 is None:
        psi = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
        inst.init_uniform(psi)
    else:
        psi = to_gpu(torch, psi0)
    inst.evolve(psi, T, K)
    obs = inst.observables(psi)
    return inst, psi, obs


EVOLVE_CASES = [
    # (n, source, T, K)
    (1, "unit", 3.0, 30),
    (2, "rand", 3.0, 25),
    (3, "planted", 4.0, 40),
    (5, "planted", 5.0, 50),
    (6, "paper", 8.0, 80),
    (9, "planted", 5.0, 50),
    (10, "planted", 5.0, 50),
    (12, "planted", 20.0, 400),   # the n=12 configuration: T=20, dt=0.05
    (14, "planted", 3.0, 30),
    (15, "planted", 3.0, 20),     # strided width 5
    (16, "planted", 3.0, 20),     # width 6
    (17, "planted", 3.0, 12),     # width 7
    (18, "planted", 2.0, 8),      # width 8
    (19, "planted", 2.0, 8),      # width 9
    (20, "planted20", 10.0, 200), # the n=20 configuration, T=10, dt=0.05
    (21, "planted", 1.0, 4),      # one 11-bit strided group (2 round trips per step)
]


def instance_for(n, src):
    if src == "unit":
        return [[1]]
    if src == "rand":
        return satgen.random_instance(n, 3, seed=n, width=2)
    if src == "paper":
        return paper_instance()[1]
    if src == "planted20":
        return satgen.load_instance("planted_n20_s0")["clauses"]
    return satgen.planted_instance(n, 11)["clauses"]


@pytest.mark.parametrize("n,src,T,K", EVOLVE_CASES, ids=[f"n{c[0]}-{c[1]}-K{c[3]}" for c in EVOLVE_CASES])
def test_evolve_matches_oracle_strang(q, torch, n, src, T, K):
    cl = instance_for(n, src)
    e = oracle.violated_counts(n, cl)
    ref = oracle.evolve_strang(n, cl, T, K, energies=e)
    _, psi, obs = run_gpu(q, torch, n, cl, T, K)
    got = to_np(psi)
    err = np.max(np.abs(got - ref))
    assert err <= AMP_TOL, err
    p_ref = oracle.success_prob(ref, e)
    assert abs(obs["ground_prob"] - p_ref) <= PROB_TOL, (obs, p_ref)
    assert abs(obs["ground_prob"] / obs["norm"] - p_ref) <= PROB_TOL, (obs, p_ref)
    assert abs(obs["norm"] - 1.0) <= NORM_TOL
    assert obs["ground_count"] == int(np.count_nonzero(e == 0))


def test_evolve_from_arbitrary_state(q, torch):
    n, T, K = 16, 2.5, 10
    cl = satgen.planted_instance(n, 3)["clauses"]
    rng = np.random.default_rng(0)
    psi0 = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    psi0 /= np.sqrt(oracle.norm(psi0))
    psi0 = psi0.astype(np.complex64).astype(np.complex128)
    ref = oracle.evolve_strang(n, cl, T, K, psi0=psi0)
    _, psi, _ = run_gpu(q, torch, n, cl, T, K, psi0=psi0)
    assert np.max(np.abs(to_np(psi) - ref)) <= AMP_TOL


@pytest.mark.parametrize("n", [8, 17])
def test_evolve_range_composes(q, torch, n):
    cl = satgen.planted_instance(n, 4)["clauses"]
    T, K = 4.0, 24
    inst = q.Instance(n, cl)
    a = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    inst.init_uniform(a)
    b = a.clone()
    inst.evolve(a, T, K)
    for k0, k1 in [(0, 7), (7, 7), (7, 20), (20, 24)]:
        inst.evolve_range(b, T, K, k0, k1)
    ref = oracle.evolve_strang(n, cl, T, K)
    assert np.max(np.abs(to_np(a) - to_np(b))) <= AMP_TOL
    assert np.max(np.abs(to_np(b) - ref)) <= AMP_TOL


def rabi_closed_form(s, t, psi0):
    a, b = 1.0 - s, s
    c, om = 0.5 * (a + b), 0.5 * np.hypot(a, b)
    X = np.array([[0, 1], [1, 0]], dtype=complex)
    Z = np.diag([1.0, -1.0]).astype(complex)
    M = 0.5 * (-a * X + b * Z)
    U = np.exp(-1j * c * t) * (np.cos(om * t) * np.eye(2) - 1j * np.sin(om * t) * M / om)
    return U @ psi0


def test_frozen_schedule_one_qubit_rabi(q, torch):
    # Constant s: Strang converges to the closed-form propagator at second order.
    s, T = 0.4, 5.0
    psi0 = np.array([0.6, 0.8j])
    ref = rabi_closed_form(s, T, psi0)
    errs = []
    for K in (20, 40, 80):
        inst = q.Instance(1, [[1]])
        psi = to_gpu(torch, psi0)
        inst.evolve_schedule(psi, T / K, [s] * K)
        got = to_np(psi)
        assert np.max(np.abs(got - oracle.evolve_strang(1, [[1]], T, K, psi0=psi0, s_values=[s] * K))) <= AMP_TOL
        errs.append(np.max(np.abs(got - ref)))
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5, errs


@pytest.mark.parametrize("n", [6, 20])
def test_s_zero_keeps_uniform(q, torch, n):
    cl = satgen.planted_instance(n, 2)["clauses"]
    inst = q.Instance(n, cl)
    psi = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    inst.init_uniform(psi)
    inst.evolve_schedule(psi, 0.1, [0.0] * 40)
    assert np.max(np.abs(to_np(psi) - oracle.uniform_state(n))) <= 1e-6


def test_no_clauses_keeps_uniform(q, torch):
    n = 18
    _, psi, obs = run_gpu(q, torch, n, [], 10.0, 50)
    assert np.max(np.abs(to_np(psi) - oracle.uniform_state(n))) <= 1e-6
    assert obs["ground_count"] == 1 << n


# ---------------------------------------------------------------- observables
# n = 22 and 24: two strided correlation groups (6 + 6, 7 + 7 bits)
@pytest.mark.parametrize("n", [1, 3, 10, 12, 17, 21, 22, 24])
def test_observables_match_oracle(q, torch, n):
    cl = satgen.random_instance(n, 4 * n, seed=n, width=min(3, n))
    e = oracle.violated_counts(n, cl)
    rng = np.random.default_rng(n)
    psi0 = (rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)).astype(np.complex64)
    psi0 = psi0.astype(np.complex128)
    inst = q.Instance(n, cl)
    psi = to_gpu(torch, psi0)
    o = inst.observables(psi)
    assert o["norm"] == pytest.approx(oracle.norm(psi0), rel=1e-12)
    assert o["expect_hp"] == pytest.approx(oracle.expect_hp(psi0, e), rel=1e-12)
    # norm, <H_P>, ground probability: exact FP64 products, FP64 sums (1e-12).
    # <H_B>: its pair products are summed in FP32 per thread-tile (<= 320 terms),
    # then in FP64 -- 1e-7 relative.
    assert o["expect_hb"] == pytest.approx(oracle.expect_hb(n, psi0), rel=1e-7, abs=1e-9)
    assert o["ground_prob"] == pytest.approx(oracle.success_prob(psi0, e), rel=1e-12, abs=1e-300)
    assert o["ground_count"] == int(np.count_nonzero(e == 0))
    s = 0.37
    assert inst.energy(psi, s) == pytest.approx(oracle.energy(n, psi0, e, s), rel=1e-7)
    assert inst.success_prob(psi) == o["ground_prob"]
    assert inst.norm(psi) == o["norm"]
    # fixed reduction order: bit-identical on repeat
    assert inst.observables(psi) == o


# ------------------------------------------------ tensor-core WHT variant ---
# BF16x3 (hi + mid + lo, FP32 accumulation; hi and the small parts in separate
# accumulators) is held to the FP32 bar; BF16x2 to the BF16-split bar of 1e-3.
# Measured at n = 20, T = 10, 200 steps: 6.1e-7 (x3) and 2.4e-5 (x2).
TC_CASES = [(15, 3.0, 20), (17, 3.0, 12), (20, 10.0, 200), (21, 1.0, 4)]


# The BF16x2 ablation's per-step rounding is ~2^-16, so the norm left by its
# last step (after the fold of the step before) is held to 1e-5.
@pytest.mark.parametrize("kind,amp_tol,prob_tol,norm_tol", [(1, AMP_TOL, PROB_TOL, NORM_TOL), (2, 1e-3, 1e-4, 1e-5)],
                         ids=["bf16x3", "bf16x2"])
@pytest.mark.parametrize("n,T,K", TC_CASES, ids=[f"n{c[0]}-K{c[2]}" for c in TC_CASES])
def test_tensor_core_variant_matches_oracle(q, torch, kind, amp_tol, prob_tol, norm_tol, n, T, K):
    cl = satgen.load_instance("planted_n20_s0")["clauses"] if n == 20 else satgen.planted_instance(n, 11)["clauses"]
    e = oracle.violated_counts(n, cl)
    ref = oracle.evolve_strang(n, cl, T, K, energies=e)
    inst = q.Instance(n, cl)
    inst.set_variant(kind)
    assert "tensor-core" in inst.describe_plan()
    psi = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    inst.init_uniform(psi)
    inst.evolve(psi, T, K)
    o = inst.observables(psi)
    assert np.max(np.abs(to_np(psi) - ref)) <= amp_tol
    assert abs(o["ground_prob"] - oracle.success_prob(ref, e)) <= prob_tol
    assert abs(o["ground_prob"] / o["norm"] - oracle.success_prob(ref, e)) <= prob_tol
    assert abs(o["norm"] - 1.0) <= norm_tol


# ------------------------------------------------ rotation form (variant 3) ---
# exp(-i theta H_B) applied as its n one-qubit factors: the same Strang step as
# the W B W form, so the same FP32 bar against the oracle.  Cases span every
# strided width (5..10), two and three strided groups, ragged widths and a
# sub-range that starts and ends inside the run.
ROT_CASES = [(15, 3.0, 20), (16, 3.0, 20), (17, 3.0, 12), (18, 2.0, 8), (19, 2.0, 8), (20, 10.0, 200),
             (21, 1.0, 4), (22, 1.0, 5), (24, 1.0, 3)]


@pytest.mark.parametrize("n,T,K", ROT_CASES, ids=[f"n{c[0]}-K{c[2]}" for c in ROT_CASES])
def test_rotation_form_matches_oracle(q, torch, n, T, K):
    cl = satgen.load_instance("planted_n20_s0")["clauses"] if n == 20 else satgen.planted_instance(n, 11)["clauses"]
    e = oracle.violated_counts(n, cl)
    ref = oracle.evolve_strang(n, cl, T, K, energies=e)
    inst = q.Instance(n, cl)
    inst.set_variant(3)
    assert "rotation form" in inst.describe_plan()
    psi = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    inst.init_uniform(psi)
    inst.evolve(psi, T, K)
    o = inst.observables(psi)
    assert np.max(np.abs(to_np(psi) - ref)) <= AMP_TOL
    assert abs(o["ground_prob"] - oracle.success_prob(ref, e)) <= PROB_TOL
    assert abs(o["ground_prob"] / o["norm"] - oracle.success_prob(ref, e)) <= PROB_TOL
    assert abs(o["norm"] - 1.0) <= NORM_TOL
    inst.close()


def test_rotation_form_range_composes(q, torch):
    n, T, K = 19, 3.0, 30
    cl = satgen.planted_instance(n, 4)["clauses"]
    e = oracle.violated_counts(n, cl)
    ref = oracle.evolve_strang(n, cl, T, K, energies=e)
    inst = q.Instance(n, cl)
    inst.set_variant(3)
    psi = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    inst.init_uniform(psi)
    for k0, k1 in ((0, 1), (1, 17), (17, 29), (29, 30)):
        inst.evolve_range(psi, T, K, k0, k1)
    assert np.max(np.abs(to_np(psi) - ref)) <= AMP_TOL
    inst.close()


@pytest.fixture(scope="module")
def n20_reference():
    n, T, K = 20, 1.0, 4
    cl = satgen.load_instance("planted_n20_s0")["clauses"]
    e = oracle.violated_counts(n, cl)
    return n, T, K, cl, oracle.evolve_strang(n, cl, T, K, energies=e)


@pytest.mark.parametrize("variant", [0, 3], ids=["wbw", "rotation"])
@pytest.mark.parametrize("qbits,groups", [(5, 2), (7, 2), (10, 1), (11, 1)])
def test_qubits_per_pass_choice(q, torch, n20_reference, variant, qbits, groups):
    """set_variant(kind, q): the fewest strided groups of at most q bits (10
    strided bits at n = 20: 5+5 or one group); the same evolution within the FP32 bar."""
    n, T, K, cl, ref = n20_reference
    inst = q.Instance(n, cl)
    inst.set_variant(variant, qbits)
    d = inst.describe_plan()
    assert d.count("group bits") == groups, d
    psi = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    inst.init_uniform(psi)
    inst.evolve(psi, T, K)
    assert np.max(np.abs(to_np(psi) - ref)) <= AMP_TOL
    inst.close()
    with q.Instance(24, [[1, 2, 3]]) as other:
        with pytest.raises(q.QaaError):
            other.set_variant(3, 5)  # 14 strided bits: no split into groups of exactly 5


def test_variant_argument_checks(q, torch):
    inst = q.Instance(16, [[1, 2, 3]])
    with pytest.raises(q.QaaError):
        inst.set_variant(4)
    with pytest.raises(q.QaaError):
        inst.set_variant(0, 4)
    with pytest.raises(q.QaaError):
        inst.set_variant(1, 11)  # no 11-bit tensor-core tiles
