"""qaa_observables_noalloc: observables for callers that cannot allocate device memory.

Some callers of this library cannot call cudaMalloc: their device memory is
owned by another allocator (a framework's pool, a budget fixed at start-up), or
they run loops in which the device-wide synchronisation that cudaMalloc and
cudaFree may cause is not acceptable.  They cannot create a handle, so they
call this entry point with the instance itself; its scratch is a static device
array.  This file checks, through the C ABI, that two calls in a row give the
same observables as the handle-based qaa_observables, and that requests above
the static capacity are refused with a clear message.
"""

import ctypes

import numpy as np
import pytest

import satgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1103_1399_gb300 as q
    return q, torch


def noalloc_observables(q, n, clauses, psi):
    buf, m = q.flatten_clauses(clauses)
    out = q.Obs()
    st = q.lib.qaa_observables_noalloc(n, ctypes.cast(buf, ctypes.c_void_p), m, psi.data_ptr(), None,
                                       ctypes.byref(out))
    assert st == 0, q.lib.qaa_last_error().decode()
    return {"norm": out.norm, "expect_hp": out.expect_hp, "expect_hb": out.expect_hb,
            "ground_prob": out.ground_prob, "ground_count": int(out.ground_count)}


def random_state(torch, n, seed):
    rng = np.random.default_rng(seed)
    v = (rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)).astype(np.complex64)
    return torch.from_numpy(v).cuda()


def assert_close(got, ref):
    # the tolerances of the observables parity test
    assert got["norm"] == pytest.approx(ref["norm"], rel=1e-12)
    assert got["expect_hp"] == pytest.approx(ref["expect_hp"], rel=1e-12)
    assert got["expect_hb"] == pytest.approx(ref["expect_hb"], rel=1e-10, abs=1e-9)
    assert got["ground_prob"] == pytest.approx(ref["ground_prob"], rel=1e-12, abs=1e-300)
    assert got["ground_count"] == ref["ground_count"]


def test_two_calls_in_a_row_match_the_handle_path(env):
    q, torch = env
    # n = 17: correlation passes above bit 10; n = 12: the plain correlation
    # kernel; n = 6: one partial tile (amplitudes beyond 2^n masked), no pass
    # above bit 10; m = 0: no clause upload, every E(x) = 0
    cases = [(17, satgen.random_instance(17, 80, seed=21), 1),
             (12, satgen.planted_instance(12, 3)["clauses"], 2),
             (6, satgen.random_instance(6, 9, seed=5), 3),
             (12, [], 4)]
    for n, clauses, seed in cases:
        psi = random_state(torch, n, seed)
        with q.Instance(n, clauses) as inst:
            ref = inst.observables(psi)
        torch.cuda.synchronize()
        first = noalloc_observables(q, n, clauses, psi)
        second = noalloc_observables(q, n, clauses, psi)
        assert_close(first, ref)
        assert_close(second, ref)


def test_requests_above_the_static_capacity_are_refused(env):
    q, torch = env
    psi = random_state(torch, 4, 0)
    flat = (ctypes.c_int32 * (3 * 1024))(*([1, 2, 3] * 1024))
    out = q.Obs()
    st = q.lib.qaa_observables_noalloc(4, ctypes.cast(flat, ctypes.c_void_p), 1024, psi.data_ptr(), None,
                                       ctypes.byref(out))
    assert st == -1
    assert "static clause capacity" in q.lib.qaa_last_error().decode()
