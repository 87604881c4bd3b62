"""The autotuner (qaa_autotune): it times candidate pass plans on the GPU,
keeps the fastest for the handle and records it for later handles and server
requests of the same n.  A tuned plan must still match the oracle (plans differ
only in butterfly order, so within the FP32 bar), and a server request then
runs the same plan: its result equals the handle API's bit for bit."""

import time

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
    yield q, torch
    q.forget_tuned_plans()


def chosen(report):
    line = [ln for ln in report.splitlines() if ln.startswith("chosen")]
    assert len(line) == 1, report
    return line[0].split(": ", 1)[1]


@pytest.mark.parametrize("n", [16, 21])
def test_autotune_picks_a_timed_plan_and_records_it(env, n):
    q, torch = env
    cl = satgen.planted_instance(n, 3)["clauses"]
    psi = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    try:
        with q.Instance(n, cl) as inst:
            rep = inst.autotune(psi, steps=2, budget_ms=30000)
            plan = chosen(rep)
            assert inst.describe_plan() == plan
            timed = [ln.split("ms/step", 1)[1].strip() for ln in rep.splitlines() if "ms/step" in ln and not ln.startswith("chosen")]
            assert plan in timed
            assert len(timed) >= len(q.tune_candidates(n))  # stage 1 ran in full within the budget
            # the tuned plan still matches the oracle
            K, T = 12, 1.2
            inst.init_uniform(psi)
            inst.evolve(psi, T, K)
            got = psi.cpu().numpy().astype(np.complex128)
        ref = oracle.evolve_strang(n, cl, T, K)
        assert np.max(np.abs(got - ref)) <= 1e-5
        with q.Instance(n, cl) as other:
            assert other.describe_plan() == plan  # recorded for later handles of this n
    finally:
        q.forget_tuned_plans()
    with q.Instance(n, cl) as fresh:
        default = fresh.describe_plan()
    assert default == q.tune_candidates(n)[0]  # forgotten: back to the default plan


def test_server_uses_the_tuned_plan(env, monkeypatch):
    q, torch = env
    monkeypatch.setenv("QAA_PERSIST_MAX_BITS", "0")  # streamed: the request runs the plan's passes
    n, K, T = 20, 20, 2.0
    cl = satgen.planted_instance(n, 8)["clauses"]
    psi = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    try:
        with q.Instance(n, cl) as inst:
            inst.autotune(psi, steps=2, budget_ms=20000)
            inst.init_uniform(psi)
            inst.evolve(psi, T, K)
            ref = inst.observables(psi)
        with q.Server(max_slots=4) as srv:
            t = srv.submit(n, cl, T, K)
            t0 = time.time()
            while (r := srv.poll(t)) is None:
                assert time.time() - t0 < 60
                time.sleep(0.002)
        assert r["status"] == 0
        assert r["success_prob"] == ref["ground_prob"] and r["norm"] == ref["norm"]
    finally:
        q.forget_tuned_plans()


def test_autotune_on_chip_sizes_and_arguments(env):
    q, torch = env
    with q.Instance(12, [[1, 2, 3]]) as inst:
        psi = torch.empty(1 << 12, dtype=torch.complex64, device="cuda")
        assert "no pass plan" in inst.autotune(psi)
    with q.Instance(15, [[1, 2, 3]]) as inst:
        psi = torch.empty(1 << 15, dtype=torch.complex64, device="cuda")
        with pytest.raises(q.QaaError):
            inst.autotune(psi, steps=0)
        with pytest.raises(q.QaaError):
            inst.autotune(psi, steps=65)
