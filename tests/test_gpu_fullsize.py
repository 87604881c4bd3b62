"""Parity at the benchmark size (n = 30, 8 GiB state), in the launch configuration
bench.py times, on outputs the oracle can compute one by one.

* Product instance: with one-literal clauses only, E(x) = sum_i e_i(x_i) and
  every factor of the Strang step factorises over qubits, so each amplitude is
  a product of one-qubit Strang states (oracle.one_qubit_strang, complex128).
  This checks every streaming pass and both phases at full size.
* Planted instance of the benchmark: E(x) bit exact on sampled x
  (oracle.energy_at), exactly one zero-energy assignment and it is the planted
  one (two independent routes: the generator's uniqueness proof and the GPU
  count), norm conservation after the 400-step benchmark schedule.
* Plan invariance: the split-group and contiguous-group pass plans agree.
* The rotation form (variant 3) on the product instance, same schedule.

Amplitudes at n = 30 are ~2^-15, so the bar is stated relative to the largest
amplitude of the reference over all x (closed form for a product state):
max |d psi_x| over the sample <= REL_TOL * max_x |psi_x|.
"""

import os

import numpy as np
import pytest

import oracle
import satgen

pytestmark = pytest.mark.gpu

N = 30
T, DT = 40.0, 0.1
K = 400
# relative amplitude bar at n = 30: FP32 rounding grows ~ sqrt(steps x stages);
# 1e-5 relative to the largest amplitude is the n = 20 absolute bar rescaled.
REL_TOL = 1e-5
NORM_TOL = 1e-6


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1103_1399_gb300 as q
    return q, torch


def product_instance(seed=0):
    rng = np.random.default_rng(seed)
    clauses = []
    for v in range(1, N + 1):
        for _ in range(int(rng.integers(0, 3))):
            clauses.append([v if rng.integers(0, 2) else -v])
    return clauses


def gather(torch, psi, xs):
    idx = torch.as_tensor(np.asarray(xs, dtype=np.int64), device=psi.device)
    return psi[idx].cpu().numpy().astype(np.complex128)


@pytest.fixture(scope="module")
def state(env):
    q, torch = env
    psi = torch.empty(1 << N, dtype=torch.complex64, device="cuda")
    yield psi
    del psi
    torch.cuda.empty_cache()


def evolve_product(q, torch, psi, clauses, steps):
    inst = q.Instance(N, clauses)
    inst.init_uniform(psi)
    inst.evolve(psi, DT * steps, steps)
    o = inst.observables(psi)
    inst.close()
    return o


def product_reference(clauses, steps, xs):
    factors = []
    for i in range(1, N + 1):
        e0 = sum(1 for c in clauses if c == [i])
        e1 = sum(1 for c in clauses if c == [-i])
        factors.append(oracle.one_qubit_strang(e0, e1, DT * steps, steps))
    out = np.ones(len(xs), dtype=np.complex128)
    for i in range(N):
        bits = (np.asarray(xs) >> i) & 1
        out *= np.where(bits == 1, factors[i][1], factors[i][0])
    return out


def product_max_amplitude(clauses, steps):
    """The reference's largest |psi_x| over all 2^30 x: the product over qubits of
    the larger one-qubit amplitude (the bar below is relative to it)."""
    out = 1.0
    for i in range(1, N + 1):
        e0 = sum(1 for c in clauses if c == [i])
        e1 = sum(1 for c in clauses if c == [-i])
        f = oracle.one_qubit_strang(e0, e1, DT * steps, steps)
        out *= max(abs(f[0]), abs(f[1]))
    return out


def product_ground_count(clauses):
    # E(x) = sum_i e_i(x_i) = 0 needs e_i(x_i) = 0 for every i
    count = 1
    for i in range(1, N + 1):
        e0 = sum(1 for c in clauses if c == [i])
        e1 = sum(1 for c in clauses if c == [-i])
        count *= (e0 == 0) + (e1 == 0)
    return count


def test_product_instance_full_size(env, state):
    q, torch = env
    clauses = product_instance(1)
    o = evolve_product(q, torch, state, clauses, K)
    rng = np.random.default_rng(7)
    xs = rng.integers(0, 1 << N, size=4000)
    ref = product_reference(clauses, K, xs)
    got = gather(torch, state, xs)
    scale = product_max_amplitude(clauses, K)
    err = np.max(np.abs(got - ref)) / scale
    assert err <= REL_TOL, err
    assert abs(o["norm"] - 1.0) <= NORM_TOL
    assert o["ground_count"] == product_ground_count(clauses)


def test_planted_benchmark_instance(env, state):
    q, torch = env
    inst_d = satgen.load_instance("planted_n30_s0")
    cl = inst_d["clauses"]
    inst = q.Instance(N, cl)
    diag = torch.empty(1 << N, dtype=torch.int16, device="cuda")
    inst.hp_diagonal(diag)
    rng = np.random.default_rng(3)
    xs = np.concatenate([rng.integers(0, 1 << N, size=300), [inst_d["planted"], 0, (1 << N) - 1]])
    got = diag[torch.as_tensor(xs, device="cuda")].cpu().numpy().view(np.uint16).astype(np.int64)
    ref = np.array([oracle.energy_at(N, cl, int(x)) for x in xs])
    assert np.array_equal(got, ref)
    assert int((diag == 0).sum().item()) == 1
    del diag
    inst.init_uniform(state)
    inst.evolve(state, T, K)
    o = inst.observables(state)
    assert o["ground_count"] == 1
    assert abs(o["norm"] - 1.0) <= NORM_TOL
    assert 0.0 <= o["ground_prob"] <= 1.0
    inst.close()


def test_pass_plans_agree(env, state):
    q, torch = env
    clauses = product_instance(2)
    steps = 20
    rng = np.random.default_rng(11)
    xs = rng.integers(0, 1 << N, size=4000)
    results = []
    for split in ("0", "1"):
        old = os.environ.get("QAA_SPLIT_GROUPS")
        os.environ["QAA_SPLIT_GROUPS"] = split
        try:
            evolve_product(q, torch, state, clauses, steps)
        finally:
            if old is None:
                del os.environ["QAA_SPLIT_GROUPS"]
            else:
                os.environ["QAA_SPLIT_GROUPS"] = old
        results.append(gather(torch, state, xs))
    ref = product_reference(clauses, steps, xs)
    scale = product_max_amplitude(clauses, steps)
    for got in results:
        assert np.max(np.abs(got - ref)) / scale <= REL_TOL
    assert np.max(np.abs(results[0] - results[1])) / scale <= REL_TOL


def test_rotation_form_full_size(env, state):
    """The rotation form (variant 3) on the full-size product instance, the
    400-step benchmark schedule: 3 HBM round trips per step."""
    q, torch = env
    clauses = product_instance(3)
    inst = q.Instance(N, clauses)
    inst.set_variant(3)
    assert "3 HBM round trips per step" in inst.describe_plan()
    inst.init_uniform(state)
    inst.evolve(state, DT * K, K)
    o = inst.observables(state)
    inst.close()
    rng = np.random.default_rng(13)
    xs = rng.integers(0, 1 << N, size=4000)
    ref = product_reference(clauses, K, xs)
    got = gather(torch, state, xs)
    scale = product_max_amplitude(clauses, K)
    assert np.max(np.abs(got - ref)) / scale <= REL_TOL
    assert abs(o["norm"] - 1.0) <= NORM_TOL
    assert o["ground_count"] == product_ground_count(clauses)


def test_plan_description(env):
    q, _ = env
    with q.Instance(N, [[1, 2, 3]]) as inst:
        d = inst.describe_plan()
    assert d.startswith("streaming") and "rotation form" in d and "3 HBM round trips per step" in d
    with q.Instance(N, [[1, 2, 3]]) as inst:
        inst.set_variant(0)
        assert "W.B.W" in inst.describe_plan() and "4 HBM round trips per step" in inst.describe_plan()
    with q.Instance(12, [[1, 2, 3]]) as inst:
        assert inst.describe_plan().startswith("on-chip")
