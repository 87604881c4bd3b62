"""The serving loop (qaa_server_*): continuous batching of evolve requests.

* Each request's result is the same alone and in a mix of sizes served
  concurrently -- bit for bit: every request runs the same kernels in the same
  order whatever else is in flight (on-chip batches, one CTA per request;
  mid-size requests, one persistent launch each).  It also agrees with the
  handle API (qaa_create + evolve + observables) within the FP32 tolerance
  (mid-size requests there use other tile shapes, hence other rounding).
* Admission by device memory: with an arena that holds only a few states at a
  time every request still completes, later ones admitted as memory frees up.
* A request that can never fit is refused at submission (QAA_E_NOMEM), not
  left waiting; a queued request can be cancelled; a host-side injected
  failure or delay disturbs no other request.
"""

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
    return q, torch


def alone(q, torch, n, cl, T, K):
    with q.Instance(n, cl) as inst:
        psi = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
        inst.init_uniform(psi)
        inst.evolve(psi, T, K)
        return inst.observables(psi)


def wait_all(srv, tickets, timeout=120.0):
    out, t0 = {}, time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = srv.poll(t)
                if r is not None:
                    out[t] = r
        assert time.time() - t0 < timeout, "requests did not finish"
        time.sleep(0.002)
    return out


MIX = [(10, 1, 2.0, 40), (12, 2, 5.0, 100), (13, 3, 1.0, 20), (14, 4, 2.5, 50), (15, 5, 2.0, 40),
       (16, 6, 1.5, 30), (18, 7, 1.0, 20), (20, 8, 1.0, 20), (11, 9, 3.0, 60), (17, 10, 2.0, 40)]


def test_same_result_alone_and_in_the_mix(env):
    q, torch = env
    insts = {seed: satgen.planted_instance(n, seed)["clauses"] for n, seed, _, _ in MIX}
    with q.Server(max_slots=64) as srv:
        tickets = [srv.submit(n, insts[seed], T, K) for n, seed, T, K in MIX]
        res = wait_all(srv, tickets)
        stats = srv.stats()
    keys = ("success_prob", "norm", "energy", "expect_hb", "ground_count")
    for (n, seed, T, K), t in zip(MIX, tickets):
        r = res[t]
        assert r["status"] == 0
        with q.Server(max_slots=4) as one:
            solo = next(iter(wait_all(one, [one.submit(n, insts[seed], T, K)]).values()))
        assert all(r[k] == solo[k] for k in keys), (n, r, solo)
        ref = alone(q, torch, n, insts[seed], T, K)
        assert abs(r["success_prob"] - ref["ground_prob"]) <= 1e-6
        assert abs(r["norm"] - ref["norm"]) <= 1e-6
        assert r["ground_count"] == ref["ground_count"] == 1
        assert r["t_submit"] <= r["t_admit"] <= r["t_done"]
    assert stats["batched_requests"] == sum(1 for n, *_ in MIX if n <= 14)
    assert stats["streamed_requests"] == sum(1 for n, *_ in MIX if n > 14)


def test_streamed_requests_as_launch_graphs_are_bit_identical(env, monkeypatch):
    """QAA_SERVER_GRAPH_BITS (read when the server is created) runs streamed
    requests up to that size as one launch graph each: the same kernels in the
    same order with the same phase rows and norm-fold slots, so the same
    results bit for bit as per-pass launches."""
    q, _ = env
    reqs = [(18, 31, 2.0, 40), (20, 32, 1.0, 19), (21, 33, 1.0, 9)]
    insts = {seed: satgen.planted_instance(n, seed)["clauses"] for n, seed, _, _ in reqs}
    keys = ("success_prob", "norm", "energy", "expect_hb", "ground_count")

    def serve():
        with q.Server(max_slots=8) as srv:
            tickets = [srv.submit(n, insts[seed], T, K) for n, seed, T, K in reqs]
            res = wait_all(srv, tickets)
        return [res[t] for t in tickets]

    monkeypatch.delenv("QAA_SERVER_GRAPH_BITS", raising=False)
    plain = serve()
    monkeypatch.setenv("QAA_SERVER_GRAPH_BITS", "22")
    graphs = serve()
    for a, b in zip(plain, graphs):
        assert a["status"] == b["status"] == 0
        assert all(a[k] == b[k] for k in keys), (a, b)


@pytest.mark.parametrize("n,T,K", [(15, 3.0, 20), (16, 2.0, 16), (19, 2.0, 8), (21, 1.0, 4)])
def test_persistent_requests_match_oracle(env, n, T, K, monkeypatch):
    q, _ = env
    monkeypatch.setenv("QAA_PERSIST_MAX_BITS", "24")  # every size the persistent kernel takes
    cl = satgen.planted_instance(n, 13)["clauses"]
    e = oracle.violated_counts(n, cl)
    ref = oracle.evolve_strang(n, cl, T, K, energies=e)
    with q.Server(max_slots=4) as srv:
        r = next(iter(wait_all(srv, [srv.submit(n, cl, T, K)]).values()))
    assert r["status"] == 0
    assert abs(r["success_prob"] - oracle.success_prob(ref, e)) <= 1e-6
    assert abs(r["success_prob"] / r["norm"] - oracle.success_prob(ref, e)) <= 1e-6
    assert abs(r["norm"] - 1.0) <= 1e-6
    assert abs(r["energy"] - oracle.expect_hp(ref, e)) <= 1e-4
    assert abs(r["expect_hb"] - oracle.expect_hb(n, ref)) <= 1e-4


def test_batched_result_matches_oracle(env):
    q, _ = env
    n, T, K = 11, 4.0, 80
    cl = satgen.planted_instance(n, 21)["clauses"]
    e = oracle.violated_counts(n, cl)
    ref = oracle.evolve_strang(n, cl, T, K, energies=e)
    with q.Server(max_slots=8) as srv:
        r = wait_all(srv, [srv.submit(n, cl, T, K)])
    r = next(iter(r.values()))
    assert abs(r["success_prob"] - oracle.success_prob(ref, e)) <= 1e-6
    assert abs(r["success_prob"] / r["norm"] - oracle.success_prob(ref, e)) <= 1e-6
    assert abs(r["energy"] - oracle.expect_hp(ref, e)) <= 1e-5
    assert abs(r["expect_hb"] - oracle.expect_hb(n, ref)) <= 1e-5


def test_admission_under_a_small_budget(env):
    q, torch = env
    n, T, K = 18, 1.0, 20
    cl = satgen.planted_instance(n, 31)["clauses"]
    budget = 6 << 20  # room for two n = 18 requests (2 MiB state + tables) at a time
    with q.Server(hbm_budget_bytes=budget, max_slots=64) as srv:
        tickets = [srv.submit(n, cl, T, K) for _ in range(8)]
        res = wait_all(srv, tickets)
        stats = srv.stats()
    assert all(r["status"] == 0 for r in res.values())
    assert stats["peak_used_bytes"] <= stats["arena_bytes"] <= budget + 256
    admits = sorted(r["t_admit"] for r in res.values())
    dones = sorted(r["t_done"] for r in res.values())
    assert admits[-1] > dones[0]  # the last admissions waited for earlier completions
    first = next(iter(res.values()))
    assert all(r["success_prob"] == first["success_prob"] for r in res.values())
    ref = alone(q, torch, n, cl, T, K)
    assert abs(first["success_prob"] - ref["ground_prob"]) <= 1e-6


def test_request_that_can_never_fit_is_refused(env):
    q, _ = env
    with q.Server(hbm_budget_bytes=4 << 20, max_slots=4) as srv:
        with pytest.raises(q.QaaError) as ei:
            srv.submit(20, [[1, 2, 3]], 1.0, 10)  # 8 MiB state
        assert ei.value.status == -2
        r = wait_all(srv, [srv.submit(12, [[1, 2, 3]], 1.0, 10)])
        assert next(iter(r.values()))["status"] == 0


def test_cancel_and_injected_faults_leave_others_intact(env):
    q, torch = env
    n, T, K = 16, 1.0, 20
    cl = satgen.planted_instance(n, 41)["clauses"]
    ref = alone(q, torch, n, cl, T, K)
    with q.Server(hbm_budget_bytes=2 << 20, max_slots=2) as srv:
        srv.inject(1, 50)  # the worker stalls for 50 ms once
        tickets = [srv.submit(n, cl, T, K) for _ in range(6)]
        srv.cancel(tickets[-1])  # still queued behind the stalled worker
        srv.inject(2)  # fail the next admitted request only
        res = wait_all(srv, tickets)
        with pytest.raises(q.QaaError):
            srv.cancel(tickets[0])  # already finished
    statuses = [res[t]["status"] for t in tickets]
    assert statuses[-1] == -6  # cancelled
    assert statuses.count(-3) == 1  # the injected failure
    ok = [res[t] for t in tickets if res[t]["status"] == 0]
    assert len(ok) == 4
    assert all(r["success_prob"] == ok[0]["success_prob"] for r in ok)
    assert abs(ok[0]["success_prob"] - ref["ground_prob"]) <= 1e-6


def test_invalid_submissions(env):
    q, _ = env
    with q.Server(max_slots=4) as srv:
        with pytest.raises(q.QaaError):
            srv.submit(5, [[1, 9, 2]], 1.0, 10)
        with pytest.raises(q.QaaError):
            srv.submit(5, [[1, 2, 3]], 1.0, 0)
        with pytest.raises(q.QaaError):
            srv.poll(12345)


def test_stuck_grid_barrier_times_out_and_the_server_recovers(env):
    """A persistent request whose grid barrier can never complete (injected)
    ends with QAA_E_TIMEOUT after the barrier's bounded wait; requests before
    and after it, on chip, persistent and streamed, finish correctly."""
    q, torch = env
    T, K = 1.0, 10
    inst = {n: satgen.planted_instance(n, 50 + n)["clauses"] for n in (12, 16, 19)}
    with q.Server(max_slots=8) as srv:
        srv.inject(3)
        bad = srv.submit(16, inst[16], T, K)
        res = wait_all(srv, [bad], timeout=120.0)
        assert res[bad]["status"] == -4
        good = [srv.submit(n, inst[n], T, K) for n in (12, 16, 19)]
        res = wait_all(srv, good, timeout=120.0)
    for n, t in zip((12, 16, 19), good):
        r = res[t]
        assert r["status"] == 0
        ref = alone(q, torch, n, inst[n], T, K)
        assert abs(r["success_prob"] - ref["ground_prob"]) <= 1e-6


def overlapping_pairs(rs):
    out = []
    for i in range(len(rs)):
        for j in range(i + 1, len(rs)):
            a, b = rs[i], rs[j]
            if max(a["t_dev_start"], b["t_dev_start"]) < min(a["t_dev_end"], b["t_dev_end"]):
                out.append((i, j))
    return out


def test_requests_overlap_on_the_device(env):
    """Requests admitted together are in flight on the GPU at the same time:
    their device intervals (device-timer stamps on the request's own stream,
    before its first copy and at the end of its observables) overlap
    -- mid-size requests run as persistent launches on disjoint SMs, larger
    ones interleave their passes on the issuer streams -- and each result is
    still the same, bit for bit, as the same request served alone."""
    q, _ = env
    reqs = [(16, 60 + i, 10.0, 200) for i in range(4)] + [(20, 70 + i, 5.0, 100) for i in range(4)]
    insts = {seed: satgen.planted_instance(n, seed)["clauses"] for n, seed, _, _ in reqs}
    with q.Server(max_slots=16) as srv:
        tickets = [srv.submit(n, insts[seed], T, K) for n, seed, T, K in reqs]
        res = wait_all(srv, tickets)
    rs = [res[t] for t in tickets]
    for r in rs:
        assert r["status"] == 0
        assert 0.0 <= r["t_dev_start"] < r["t_dev_end"]
    assert overlapping_pairs(rs[:4]), [(r["t_dev_start"], r["t_dev_end"]) for r in rs[:4]]
    assert overlapping_pairs(rs[4:]), [(r["t_dev_start"], r["t_dev_end"]) for r in rs[4:]]
    keys = ("success_prob", "norm", "energy", "expect_hb", "ground_count")
    with q.Server(max_slots=4) as one:
        for (n, seed, T, K), r in zip(reqs, rs):
            solo = next(iter(wait_all(one, [one.submit(n, insts[seed], T, K)]).values()))
            assert all(r[k] == solo[k] for k in keys), (n, r, solo)
