"""The rotation form's 12-bit low pass (kLpRot12): each warp quad holds four
consecutive 1024-amplitude tiles, rotates index bits 10..11 across them in
shared memory, then each warp rotates bits 0..9 and applies 2^-n P as the
10-bit low pass does.  It is a tuning option (QAA_LOW_BITS=12, at any n >= 17)
and an autotuner candidate for n >= 31, not the default.

* n = 17, 20, 23 (forced): one strided group of 5, 8 or 11 bits from bit
  12, against the complex128 oracle (max amplitude 1e-5, P_succ 1e-6).
* n = 20 (forced): evolve_range pieces match one evolve call up to FP32
  rounding; the launch graph gives the same states as per-pass launches bit
  for bit.
* n = 31 and 32, product instances (forced): low pass bits [0,12), two
  10-bit groups at n = 32 (recombined), 10 + 9 at n = 31, all with 128-byte
  runs, against the closed-form product of one-qubit Strang states on
  sampled amplitudes.
"""

import numpy as np
import pytest

import oracle
import satgen
from test_gpu_qbits import product_check, product_instance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1103_1399_gb300 as q
    return q, torch


@pytest.mark.parametrize("n,groups", [(17, ["[12,17)"]), (20, ["[12,17)+[17,20)"]),
                                      (23, ["[12,17)+[17,23)"])])
def test_forced_low12_matches_oracle(env, monkeypatch, n, groups):
    q, torch = env
    monkeypatch.setenv("QAA_LOW_BITS", "12")
    T, K = 2.5, 15
    cl = satgen.planted_instance(n, 50 + n)["clauses"]
    e = oracle.violated_counts(n, cl)
    ref = oracle.evolve_strang(n, cl, T, K, energies=e)
    psi = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    with q.Instance(n, cl) as inst:
        plan = inst.describe_plan()
        assert "low pass bits [0,12)" in plan, plan
        for g in groups:
            assert "group bits " + g in plan, plan
        inst.init_uniform(psi)
        inst.evolve(psi, T, K)
        o = inst.observables(psi)
    got = psi.cpu().numpy().astype(np.complex128)
    assert np.max(np.abs(got - ref)) <= 1e-5
    assert abs(o["ground_prob"] - oracle.success_prob(ref, e)) <= 1e-6
    assert abs(o["ground_prob"] / o["norm"] - oracle.success_prob(ref, e)) <= 1e-6


def test_forced_low12_ranges_and_graph(env, monkeypatch):
    q, torch = env
    monkeypatch.setenv("QAA_LOW_BITS", "12")
    n, T, K = 20, 3.0, 30
    cl = satgen.planted_instance(n, 61)["clauses"]

    def run(call, mode=0):
        with q.Instance(n, cl) as inst:
            inst.set_launch_mode(mode)
            psi = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
            inst.init_uniform(psi)
            call(inst, psi)
            torch.cuda.synchronize()
            return psi

    whole = run(lambda i, p: i.evolve(p, T, K))

    def pieces(i, p):
        for k0, k1 in ((0, 7), (7, 8), (8, 30)):
            i.evolve_range(p, T, K, k0, k1)

    split = run(pieces)
    # a split applies the two half phases at each cut separately (not merged
    # into one table entry): equal up to FP32 rounding
    assert torch.max(torch.abs(split - whole)).item() <= 1e-6
    # the launch graph runs the same kernels in the same order
    assert torch.equal(run(lambda i, p: i.evolve(p, T, K), mode=1), whole)
    assert torch.equal(run(pieces, mode=1), split)


@pytest.mark.parametrize("n,groups", [
    (31, ["group bits [12,17)+[17,22)", "group bits [22,27)+[27,31)"]),
    (32, ["group bits [12,17)+[27,32)", "group bits [17,22)+[22,27)"]),
])
def test_forced_low12_product_instances(env, monkeypatch, n, groups):
    q, torch = env
    monkeypatch.setenv("QAA_LOW_BITS", "12")
    T, K = 2.0, 16
    cl = product_instance(n, 11 + n)
    plan, err, o = product_check(q, torch, n, cl, T, K, 3)
    assert "low pass bits [0,12)" in plan and "3 HBM round trips" in plan, plan
    for g in groups:
        assert g in plan, plan
    assert "128B runs" in plan and "64B runs" not in plan, plan
    assert err <= 1e-5, (plan, err)
    assert abs(o["norm"] - 1.0) <= 1e-6


def test_low12_is_an_autotune_candidate_beyond_l2(env):
    q, _ = env
    for n in (31, 32, 34):
        descs = q.tune_candidates(n)
        assert "low pass bits [0,10)" in descs[0], descs[0]  # the default keeps the 10-bit low pass
        assert sum("low pass bits [0,12)" in d for d in descs) == 1, descs
    assert not any("low pass bits [0,12)" in d for d in q.tune_candidates(30))


def test_qubits_per_pass_that_leave_no_12_bit_split_fall_back_to_10(env, monkeypatch):
    """QAA_LOW_BITS=12 with q = 5 at n = 20: the 8 bits above a 12-bit low pass
    have no split into groups of 5..5 bits, so the plan keeps the 10-bit low
    pass (two 5-bit groups) instead of producing 4-bit groups; the evolution
    matches the oracle."""
    q, torch = env
    monkeypatch.setenv("QAA_LOW_BITS", "12")
    n, T, K = 20, 2.0, 8
    cl = satgen.planted_instance(n, 11)["clauses"]
    e = oracle.violated_counts(n, cl)
    ref = oracle.evolve_strang(n, cl, T, K, energies=e)
    psi = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    with q.Instance(n, cl) as inst:
        inst.set_variant(3, 5)
        d = inst.describe_plan()
        assert "low pass bits [0,10)" in d and d.count("group bits") == 2, d
        inst.init_uniform(psi)
        inst.evolve(psi, T, K)
        o = inst.observables(psi)
    assert np.max(np.abs(psi.cpu().numpy().astype(np.complex128) - ref)) <= 1e-5
    assert abs(o["ground_prob"] - oracle.success_prob(ref, e)) <= 1e-6
