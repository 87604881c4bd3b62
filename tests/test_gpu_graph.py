"""Launch-graph mode (qaa_set_launch_mode(h, QAA_LAUNCH_GRAPH)): one CUDA graph
per step range, a WHILE conditional node over blocks of 8 Strang steps with
the phase rows computed on the device.

The graph runs the same kernels in the same order with phase rows from the
same FP64 entry functions as the per-pass launches, so the final state must
be identical bit for bit.  Cases cover every branch of the graph's structure
(no loop iteration, no remainder, both), evolve_range sub-ranges, a
caller-supplied schedule, the two- and three-group plans and the tensor-core
variant; one case is also checked against the complex128 oracle.
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


def run(q, torch, n, cl, mode, call, variant=0):
    with q.Instance(n, cl) as inst:
        inst.set_variant(variant)
        inst.set_launch_mode(mode)
        psi = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
        inst.init_uniform(psi)
        call(inst, psi)
        torch.cuda.synchronize()
        return psi


# K - 1 merged steps = 8 L + R: (K=1: L=0 R=0), (2: 0,1), (9: 1,0), (10: 1,1), (37: 4,4)
@pytest.mark.parametrize("n", [15, 17, 20, 22])
@pytest.mark.parametrize("K", [1, 2, 9, 10, 37])
def test_graph_equals_per_pass_launches(env, n, K):
    q, torch = env
    cl = satgen.planted_instance(n, 100 + n)["clauses"]
    T = 0.15 * K
    a = run(q, torch, n, cl, 0, lambda i, p: i.evolve(p, T, K))
    b = run(q, torch, n, cl, 1, lambda i, p: i.evolve(p, T, K))
    assert torch.equal(a, b)


@pytest.mark.parametrize("n", [16, 21])
def test_graph_ranges_and_schedule(env, n):
    q, torch = env
    cl = satgen.planted_instance(n, 7)["clauses"]
    K, T = 40, 4.0

    def ranges(i, p):
        for k0, k1 in ((0, 5), (5, 23), (23, 24), (24, 40)):
            i.evolve_range(p, T, K, k0, k1)

    assert torch.equal(run(q, torch, n, cl, 0, ranges), run(q, torch, n, cl, 1, ranges))
    s = np.sort(np.random.default_rng(3).uniform(0, 1, size=19))

    def sched(i, p):
        i.evolve_schedule(p, 0.12, s)

    assert torch.equal(run(q, torch, n, cl, 0, sched), run(q, torch, n, cl, 1, sched))


def test_graph_reused_and_rebuilt(env):
    q, torch = env
    n, K, T = 18, 12, 1.5
    cl = satgen.planted_instance(n, 5)["clauses"]

    def twice(i, p):
        i.profile(True)
        i.evolve(p, T, K)
        i.evolve(p, T, K)          # same key: the graph is relaunched
        i.evolve(p, 2 * T, K + 3)  # new key: rebuilt
        prof = i.profile_read()
        i.profile(False)
        if i_mode[0] == 1:
            assert prof["graph"][0] == 3
            assert prof["strided"][0] == 0 and prof["low_merge"][0] == 0

    i_mode = [0]
    a = run(q, torch, n, cl, 0, twice)
    i_mode[0] = 1
    b = run(q, torch, n, cl, 1, twice)
    assert torch.equal(a, b)


def test_graph_tensor_core_variant(env):
    q, torch = env
    n, K, T = 19, 11, 1.1
    cl = satgen.planted_instance(n, 9)["clauses"]
    a = run(q, torch, n, cl, 0, lambda i, p: i.evolve(p, T, K), variant=1)
    b = run(q, torch, n, cl, 1, lambda i, p: i.evolve(p, T, K), variant=1)
    assert torch.equal(a, b)


@pytest.mark.parametrize("n,K", [(17, 1), (20, 10), (23, 19)])
def test_graph_rotation_form(env, n, K):
    q, torch = env
    cl = satgen.planted_instance(n, 12)["clauses"]
    a = run(q, torch, n, cl, 0, lambda i, p: i.evolve(p, 0.1 * K, K), variant=3)
    b = run(q, torch, n, cl, 1, lambda i, p: i.evolve(p, 0.1 * K, K), variant=3)
    assert torch.equal(a, b)


def test_graph_matches_oracle(env):
    q, torch = env
    n, K, T = 16, 25, 2.5
    cl = satgen.planted_instance(n, 11)["clauses"]
    e = oracle.violated_counts(n, cl)
    ref = oracle.evolve_strang(n, cl, T, K, energies=e)
    got = run(q, torch, n, cl, 1, lambda i, p: i.evolve(p, T, K)).cpu().numpy().astype(np.complex128)
    assert np.max(np.abs(got - ref)) <= 1e-5


def test_launch_mode_argument_checks(env):
    q, _ = env
    with q.Instance(15, [[1, 2, 3]]) as inst:
        with pytest.raises(q.QaaError):
            inst.set_launch_mode(2)
        inst.set_launch_mode(1)
        inst.set_launch_mode(0)


@pytest.mark.parametrize("n,K", [(16, 9), (21, 5), (24, 3)])
@pytest.mark.parametrize("variant", [0, 3], ids=["wbw", "rotation"])
def test_stored_clause_counts_are_bit_identical(env, monkeypatch, n, K, variant):
    """The merged low passes read per-tile counts stored once per handle
    (QAA_LP_COUNTS=0 recounts every step): the same E(x), the same state."""
    q, torch = env
    cl = satgen.planted_instance(n, 30 + n)["clauses"]
    a = run(q, torch, n, cl, 0, lambda i, p: i.evolve(p, 0.2 * K, K), variant=variant)
    monkeypatch.setenv("QAA_LP_COUNTS", "0")
    b = run(q, torch, n, cl, 0, lambda i, p: i.evolve(p, 0.2 * K, K), variant=variant)
    assert torch.equal(a, b)
