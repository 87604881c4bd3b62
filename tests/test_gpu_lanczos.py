"""Lowest levels of H(s) by Lanczos on the GPU (qaa_lowest_eigenvalues)
against the oracle: dense diagonalisation restricted to the sector reachable
from the uniform state (start 0), all levels (start 1, dense or sparse ARPACK
at n = 16).  Bar: 1e-8 x ||H|| (||H|| <= (1 - s) n + s m), FP64 vectors."""

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


def bar(n, m, s):
    return 1e-8 * ((1.0 - s) * n + s * m) + 1e-10


@pytest.mark.parametrize("n,src", [(10, "planted"), (12, "planted"), (12, "ratio")])
@pytest.mark.parametrize("s", [0.2, 0.5, 0.8, 1.0])
def test_sector_levels_match_dense(env, n, src, s):
    q, _ = env
    cl = satgen.planted_instance(n, 3)["clauses"] if src == "planted" else satgen.ratio_instance(n, 3, min_solutions=2)["clauses"]
    ref = oracle.sector_eigenvalues(n, cl, s, 3)
    with q.Instance(n, cl) as inst:
        got, its = inst.lowest_eigenvalues(s, k=3, max_iter=300, start=0)
    assert len(got) == len(ref), (got, ref)
    assert np.max(np.abs(np.array(got) - ref)) <= bar(n, len(cl), s), (got, ref)


def test_s_zero_uniform_start_is_one_level(env):
    q, _ = env
    cl = satgen.planted_instance(11, 1)["clauses"]
    with q.Instance(11, cl) as inst:
        got, its = inst.lowest_eigenvalues(0.0, k=3, max_iter=50, start=0)
    assert its == 1 and len(got) == 1 and abs(got[0]) <= 1e-6


@pytest.mark.parametrize("s", [0.3, 0.7])
def test_random_start_all_levels_dense(env, s):
    q, _ = env
    n = 11
    cl = satgen.ratio_instance(n, 6, min_solutions=1)["clauses"]
    lam = oracle.eigenvalues(n, cl, s)
    levels = [lam[0]]
    for v in lam[1:]:
        if v - levels[-1] > 1e-8:
            levels.append(v)
    with q.Instance(n, cl) as inst:
        got, _ = inst.lowest_eigenvalues(s, k=3, max_iter=400, start=1, seed=7)
    assert len(got) == 3
    assert np.max(np.abs(np.array(got) - np.array(levels[:3]))) <= bar(n, len(cl), s), (got, levels[:3])


def test_random_start_n16_matches_sparse(env):
    q, _ = env
    n, s = 16, 0.6
    cl = satgen.planted_instance(n, 2)["clauses"]
    ref = oracle.sparse_levels(n, cl, s, 2)
    with q.Instance(n, cl) as inst:
        got, _ = inst.lowest_eigenvalues(s, k=2, max_iter=400, start=1, seed=3)
    assert np.max(np.abs(np.array(got) - ref)) <= bar(n, len(cl), s), (got, ref)


def test_gap_scan_matches_oracle(env):
    q, _ = env
    n = 10
    cl = satgen.planted_instance(n, 5)["clauses"]
    with q.Instance(n, cl) as inst:
        for s in (0.3, 0.6, 0.9):
            got, _ = inst.lowest_eigenvalues(s, k=2, max_iter=300, start=0)
            assert abs((got[1] - got[0]) - oracle.sector_gap(n, cl, s)) <= 2 * bar(n, len(cl), s)


def test_argument_checks(env):
    q, _ = env
    with q.Instance(10, [[1, 2, 3]]) as inst:
        for kw in ({"k": 0}, {"k": 9}, {"max_iter": 1}, {"start": 2}):
            with pytest.raises(q.QaaError):
                inst.lowest_eigenvalues(0.5, **kw)
