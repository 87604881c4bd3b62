"""Random 3-SAT at the clause/variable ratio of Sec. 4.3 (~4.2, near the
satisfiability threshold), with degenerate ground states, under non-linear
schedules s(t) (qaa_evolve_schedule).  Against the complex128 oracle: max
amplitude error <= 1e-5, ground-state probability (summed over every
zero-energy assignment, Sec. 2.1) within 1e-6 of the normalised state, and the
GPU's count of zero-energy assignments equal to the brute-force count."""

import math

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


SCHEDULES = {
    # slow near both ends, where the gap of H(s) is smallest for many instances
    "sin2": lambda u: math.sin(0.5 * math.pi * u) ** 2,
    # slow near the end only
    "sqrt": lambda u: math.sqrt(u),
}


@pytest.mark.parametrize("n,T,K,seed", [(10, 6.0, 120, 1), (14, 4.0, 60, 2), (17, 3.0, 30, 3), (20, 2.0, 16, 4)])
@pytest.mark.parametrize("sched", sorted(SCHEDULES))
@pytest.mark.parametrize("variant", [0, 3], ids=["wbw", "rotation"])
def test_ratio42_degenerate_nonlinear_schedule(env, n, T, K, seed, sched, variant):
    q, torch = env
    inst_d = satgen.ratio_instance(n, seed, min_solutions=2)
    cl = inst_d["clauses"]
    dt = T / K
    s_values = [SCHEDULES[sched]((k + 0.5) / K) for k in range(K)]
    e = oracle.violated_counts(n, cl)
    ref = oracle.evolve_strang(n, cl, T, K, s_values=np.asarray(s_values), energies=e)
    psi = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    with q.Instance(n, cl) as inst:
        if n > 14:
            inst.set_variant(variant)
        elif variant:
            pytest.skip("on-chip sizes have one form")
        inst.init_uniform(psi)
        inst.evolve_schedule(psi, dt, s_values)
        o = inst.observables(psi)
    got = psi.cpu().numpy().astype(np.complex128)
    assert np.max(np.abs(got - ref)) <= 1e-5
    assert abs(o["ground_prob"] - oracle.success_prob(ref, e)) <= 1e-6
    assert abs(o["ground_prob"] / o["norm"] - oracle.success_prob(ref, e)) <= 1e-6
    assert o["ground_count"] == inst_d["solutions"] >= 2
