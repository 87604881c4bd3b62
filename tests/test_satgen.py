"""The seeded instance generator: planted, unique, deterministic."""

import os

import numpy as np
import pytest

import oracle
import satgen


@pytest.mark.parametrize("n,seed", [(6, 0), (9, 4), (12, 0), (14, 7)])
def test_planted_unique_and_checked_by_oracle(n, seed):
    inst = satgen.planted_instance(n, seed)
    e = oracle.violated_counts(n, inst["clauses"])
    assert np.flatnonzero(e == 0).tolist() == [inst["planted"]]
    # the instance is minimal: dropping the last clause leaves >1 solution
    assert oracle.count_solutions(n, inst["clauses"][:-1]) > 1
    keys = {tuple(sorted(c)) for c in inst["clauses"]}
    assert len(keys) == len(inst["clauses"])
    for c in inst["clauses"]:
        assert len({abs(l) for l in c}) == 3 and all(1 <= abs(l) <= n for l in c)


def test_deterministic_and_methods_agree():
    for n in (10, 15):
        a = satgen.planted_instance(n, 3, method="incremental")
        b = satgen.planted_instance(n, 3, method="chunked")
        assert a == b
        assert a == satgen.planted_instance(n, 3)


def test_committed_instances_are_generator_output():
    d = satgen.INSTANCE_DIR
    path = os.path.join(d, "planted_n12_s0.json")
    if not os.path.exists(path):
        pytest.skip("instances not generated")
    assert satgen.load_instance(path) == satgen.planted_instance(12, 0)
    big = satgen.load_instance(os.path.join(d, "planted_n20_s0.json"))
    assert big == satgen.planted_instance(20, 0)
    assert oracle.count_solutions(20, big["clauses"]) == 1


def test_serving_requests_shape():
    reqs = satgen.serving_requests(64, seed=0, rate=100.0)
    assert len(reqs) == 64
    arr = [r[0] for r in reqs]
    assert arr == sorted(arr)
    assert all(10 <= r[1] <= 22 and 5.0 <= r[2] <= 80.0 for r in reqs)


def test_count_solutions_matches_brute_force_energies():
    import oracle
    for n, seed in ((6, 1), (9, 2), (12, 3)):
        cl = satgen.random_instance(n, int(4.2 * n), seed)
        assert satgen.count_solutions(n, cl) == int(np.count_nonzero(oracle.violated_counts(n, cl) == 0))


def test_ratio_instance_is_deterministic_and_degenerate_when_asked():
    a = satgen.ratio_instance(14, 5, min_solutions=2)
    b = satgen.ratio_instance(14, 5, min_solutions=2)
    assert a["clauses"] == b["clauses"] and a["m"] == round(4.2 * 14)
    assert a["solutions"] >= 2
    assert all(len(set(abs(l) for l in c)) == 3 for c in a["clauses"])
    assert satgen.count_solutions(14, a["clauses"]) == a["solutions"]


def test_block_instance_structure_and_separable_energy():
    import oracle
    d = satgen.block_instance(12, 3, 20, 10, seed=4)
    assert d["m"] == 3 * 30 == len(d["clauses"])
    owner = {}
    for b, blk in enumerate(d["blocks"]):
        assert blk["vars"] == [v for v in range(1, 13) if (v - 1) % 3 == b]
        for v in blk["vars"]:
            owner[v] = b
    for lits in d["clauses"]:
        assert len({owner[abs(l)] for l in lits}) == 1  # no clause mixes blocks
        assert len({abs(l) for l in lits}) == 3
    # E(x) is the sum of the blocks' energies on their own variables
    e = oracle.violated_counts(12, d["clauses"])
    x = np.arange(1 << 12)
    total = np.zeros(1 << 12, dtype=np.int64)
    for blk in d["blocks"]:
        loc = np.zeros(1 << 12, dtype=np.int64)
        for k, v in enumerate(blk["vars"]):
            loc |= ((x >> (v - 1)) & 1) << k
        total += oracle.violated_counts(len(blk["vars"]), blk["clauses"])[loc]
    assert np.array_equal(e, total)
    # the planted assignment satisfies everything; its complement violates every repeated clause
    assert e[d["planted"]] == 0
    assert e[(1 << 12) - 1 - d["planted"]] >= 3 * 10
