"""11-qubit passes (one TMA tile of 2048 rows; the sixth bit of the second
stage is a lane bit transformed by warp shuffles).

* n = 21: a single 11-bit strided group, the default plan (2 HBM round trips
  per step), against the complex128 oracle, both forms of the H_B factor.
* n = 26, product instances: an 11-bit group as the plain pass and as the
  popcount-phase pass (QAA_GROUP_BITS=11,5 and 5,11), both forms, against the
  closed-form product of one-qubit Strang states on sampled amplitudes.
* n = 32 (32 GiB), product instance: the default plan, two 11-bit groups
  recombined as {10..14, 26..31} and {15..25}, 4 round trips per step.
"""

import numpy as np
import pytest

import oracle
import satgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1103_1399_gb300 as q
    return q, torch


def product_instance(n, seed):
    rng = np.random.default_rng(seed)
    clauses = []
    for v in range(1, n + 1):
        for _ in range(int(rng.integers(0, 3))):
            clauses.append([v if rng.integers(0, 2) else -v])
    return clauses


def factors(n, clauses, T, K):
    out = []
    for i in range(1, n + 1):
        e0 = sum(1 for c in clauses if c == [i])
        e1 = sum(1 for c in clauses if c == [-i])
        out.append(oracle.one_qubit_strang(e0, e1, T, K))
    return out


def product_check(q, torch, n, clauses, T, K, variant, samples=4000, seed=5):
    psi = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    with q.Instance(n, clauses) as inst:
        inst.set_variant(variant)
        plan = inst.describe_plan()
        inst.init_uniform(psi)
        inst.evolve(psi, T, K)
        o = inst.observables(psi)
    xs = np.random.default_rng(seed).integers(0, 1 << n, size=samples)
    idx = torch.as_tensor(xs, device="cuda")
    got = psi[idx].cpu().numpy().astype(np.complex128)
    del psi
    torch.cuda.empty_cache()
    f = factors(n, clauses, T, K)
    ref = np.ones(len(xs), dtype=np.complex128)
    scale = 1.0
    for i in range(n):
        bits = (xs >> i) & 1
        ref *= np.where(bits == 1, f[i][1], f[i][0])
        scale *= max(abs(f[i][0]), abs(f[i][1]))
    err = np.max(np.abs(got - ref)) / scale
    return plan, err, o


@pytest.mark.parametrize("variant", [0, 3], ids=["wbw", "rotation"])
def test_n21_single_eleven_bit_group_matches_oracle(env, variant):
    q, torch = env
    n, T, K = 21, 2.0, 12
    cl = satgen.planted_instance(n, 17)["clauses"]
    e = oracle.violated_counts(n, cl)
    ref = oracle.evolve_strang(n, cl, T, K, energies=e)
    psi = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    with q.Instance(n, cl) as inst:
        inst.set_variant(variant)
        assert "group bits [10,15)+[15,21)" in inst.describe_plan()
        assert "2 HBM round trips per step" in inst.describe_plan()
        inst.init_uniform(psi)
        inst.evolve(psi, T, K)
        o = inst.observables(psi)
    got = psi.cpu().numpy().astype(np.complex128)
    assert np.max(np.abs(got - ref)) <= 1e-5
    assert abs(o["ground_prob"] - oracle.success_prob(ref, e)) <= 1e-6
    assert abs(o["ground_prob"] / o["norm"] - oracle.success_prob(ref, e)) <= 1e-6


@pytest.mark.parametrize("groups", ["11,5", "5,11"])
@pytest.mark.parametrize("variant", [0, 3], ids=["wbw", "rotation"])
def test_n26_eleven_bit_plain_and_phase_passes(env, monkeypatch, groups, variant):
    q, torch = env
    monkeypatch.setenv("QAA_GROUP_BITS", groups)
    n, T, K = 26, 3.0, 30
    cl = product_instance(n, 7)
    plan, err, o = product_check(q, torch, n, cl, T, K, variant)
    assert ("[15,21)" in plan) if groups == "11,5" else ("[20,26)" in plan), plan
    assert err <= 1e-5, (plan, err)
    assert abs(o["norm"] - 1.0) <= 1e-6


@pytest.mark.parametrize("variant", [0, 3], ids=["wbw", "rotation"])
def test_n32_default_plan_two_eleven_bit_groups(env, variant):
    q, torch = env
    n, T, K = 32, 2.0, 20
    cl = product_instance(n, 9)
    plan, err, o = product_check(q, torch, n, cl, T, K, variant)
    assert "group bits [10,15)+[26,32)" in plan and "group bits [15,20)+[20,26)" in plan, plan
    assert ("4 HBM round trips" in plan) if variant == 0 else ("3 HBM round trips" in plan), plan
    assert err <= 1e-5, (plan, err)
    assert abs(o["norm"] - 1.0) <= 1e-6
