"""Fourth-order evolution (qaa_evolve_order4, Yoshida's triple jump of Strang
sub-steps) and general sub-steps (qaa_evolve_substeps) against the oracle's
fourth-order composition (oracle.evolve_order4, pinned by its dt^4
convergence) and sub-step evolution: max amplitude error <= 1e-5 (FP32), the
normalised ground probability within 1e-6.  Sizes span the on-chip evolver and
both streaming forms; the launch-graph mode must equal per-pass launches."""

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


def run(q, torch, n, cl, call, variant=0, mode=0):
    psi = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    with q.Instance(n, cl) as inst:
        if n > 14:
            inst.set_variant(variant)
        inst.set_launch_mode(mode)
        inst.init_uniform(psi)
        call(inst, psi)
        o = inst.observables(psi)
    torch.cuda.synchronize()
    return psi, o


@pytest.mark.parametrize("n,T,K", [(10, 4.0, 30), (14, 3.0, 20), (17, 2.0, 9), (20, 2.0, 6)])
@pytest.mark.parametrize("variant", [0, 3], ids=["wbw", "rotation"])
def test_order4_matches_oracle(env, n, T, K, variant):
    q, torch = env
    if n <= 14 and variant:
        pytest.skip("on-chip sizes have one form")
    cl = satgen.planted_instance(n, 21)["clauses"]
    e = oracle.violated_counts(n, cl)
    ref = oracle.evolve_order4(n, cl, T, K, energies=e)
    psi, o = run(q, torch, n, cl, lambda i, p: i.evolve_order4(p, T, K), variant)
    got = psi.cpu().numpy().astype(np.complex128)
    assert np.max(np.abs(got - ref)) <= 1e-5
    assert abs(o["ground_prob"] - oracle.success_prob(ref, e)) <= 1e-6
    assert abs(o["ground_prob"] / o["norm"] - oracle.success_prob(ref, e)) <= 1e-6


def test_order4_is_more_accurate_than_strang_at_equal_work(env):
    q, torch = env
    n, T = 12, 6.0
    cl = satgen.planted_instance(n, 5)["clauses"]
    fine = oracle.evolve_order4(n, cl, T, 200)
    p4, _ = run(q, torch, n, cl, lambda i, p: i.evolve_order4(p, T, 40))
    p2, _ = run(q, torch, n, cl, lambda i, p: i.evolve(p, T, 120))  # 120 Strang steps = 40 x 3 sub-steps
    e4 = np.max(np.abs(p4.cpu().numpy() - fine))
    e2 = np.max(np.abs(p2.cpu().numpy() - fine))
    # complex128 oracle at these sizes: 2.6e-5 against 1.7e-4
    assert e4 < 0.25 * e2, (e4, e2)


def test_substeps_random_lengths_match_oracle(env):
    q, torch = env
    n, K = 18, 11
    cl = satgen.planted_instance(n, 6)["clauses"]
    rng = np.random.default_rng(3)
    dts = rng.uniform(-0.1, 0.3, size=K)
    ss = rng.uniform(0.0, 1.0, size=K)
    ref = oracle.evolve_substeps(n, cl, dts, ss)
    for mode in (0, 1):
        psi, _ = run(q, torch, n, cl, lambda i, p: i.evolve_substeps(p, dts, ss), mode=mode)
        assert np.max(np.abs(psi.cpu().numpy().astype(np.complex128) - ref)) <= 1e-5


def test_order4_graph_equals_per_pass(env):
    q, torch = env
    n, T, K = 19, 1.5, 7
    cl = satgen.planted_instance(n, 8)["clauses"]
    a, _ = run(q, torch, n, cl, lambda i, p: i.evolve_order4(p, T, K), mode=0)
    b, _ = run(q, torch, n, cl, lambda i, p: i.evolve_order4(p, T, K), mode=1)
    assert torch.equal(a, b)


def test_substeps_argument_checks(env):
    q, torch = env
    with q.Instance(15, [[1, 2, 3]]) as inst:
        psi = torch.empty(1 << 15, dtype=torch.complex64, device="cuda")
        with pytest.raises(q.QaaError):
            inst.evolve_substeps(psi, [0.1, float("nan")], [0.2, 0.3])
        with pytest.raises(q.QaaError):
            inst.evolve_order4(psi, -1.0, 4)
