"""Pins for the oracle's violated-clause energy E(x) (Sec. 2.2 and Sec. 4.3).

The values checked here are fixed by the paper's worked example (hand-checked
facts stored in tests/golden/paper_instance.json) and by tiny instances whose
diagonals follow from the definition by inspection.  A wrong bit order, an
inverted literal sign, counting satisfied instead of violated clauses, or
dropping repeated clauses each fails at least one of them.
"""

import json
import os

import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module")
def paper(golden_dir):
    with open(os.path.join(golden_dir, "paper_instance.json")) as f:
        return json.load(f)


def test_paper_instance_has_exactly_one_solution(paper):
    # Sec. 2.2 states the proposition has only one solution.
    e = oracle.violated_counts(paper["n"], paper["clauses"])
    assert len(paper["clauses"]) == 27
    assert int(np.count_nonzero(e == 0)) == paper["paper_claim_solution_count"] == 1
    assert oracle.count_solutions(paper["n"], paper["clauses"]) == 1


def test_paper_instance_true_solution_is_index_10(paper):
    # The solution printed in Sec. 2.2 (x1..x6 = 1,1,0,1,0,0) violates the
    # clause (NOT x1 OR NOT x2 OR NOT x4); the unique solution is (0,1,0,1,0,0),
    # i.e. index 10 with x_i = bit i-1.  The hand-written certificate names a
    # true literal of every clause.
    e = oracle.violated_counts(paper["n"], paper["clauses"])
    sol = paper["true_solution"]["index"]
    assert sol == 10
    assert int(np.flatnonzero(e == 0)[0]) == sol
    bits = [(sol >> i) & 1 for i in range(6)]
    assert bits == [paper["true_solution"][f"x{i + 1}"] for i in range(6)]
    for clause, lit in zip(paper["clauses"], paper["true_solution_certificate"]):
        assert lit in clause
        assert not oracle.clause_is_violated(sol, [lit])


def test_paper_printed_solution_is_not_a_solution(paper):
    printed = paper["paper_printed_solution"]["index"]
    assert printed == 11
    e = oracle.violated_counts(paper["n"], paper["clauses"])
    assert e[printed] >= 1
    bad = paper["clauses"][paper["printed_solution_violates_clause_index"]]
    assert sorted(bad) == [-4, -2, -1]
    assert oracle.clause_is_violated(printed, bad)


def test_paper_instance_extreme_assignments(paper):
    e = oracle.violated_counts(paper["n"], paper["clauses"])
    assert e[0] == paper["energy_all_false"] == 4
    assert e[63] == paper["energy_all_true"] == 9
    for a, b in paper["duplicate_clause_pairs"]:
        assert sorted(paper["clauses"][a]) == sorted(paper["clauses"][b])


@pytest.mark.parametrize(
    "n,clauses,expected",
    [
        (2, [[1]], [1, 0, 1, 0]),            # x1 is bit 0; violated when x1 = 0
        (2, [[-2]], [0, 0, 1, 1]),           # NOT x2 violated when bit 1 set
        (3, [[1, -2, 3]], [0, 0, 1, 0, 0, 0, 0, 0]),  # only x1=0,x2=1,x3=0 (x=2)
        (1, [[1], [1]], [2, 0]),             # repeated clauses count twice
        (2, [[1, 0, 0]], [1, 0, 1, 0]),      # zero literals are padding
        (3, [], [0] * 8),                    # no clauses: zero energy
    ],
)
def test_tiny_diagonals_by_inspection(n, clauses, expected):
    assert oracle.violated_counts(n, clauses).tolist() == expected
    assert [oracle.energy_at(n, clauses, x) for x in range(1 << n)] == expected


def test_energy_at_matches_diagonal_on_random_instance():
    import satgen
    cl = satgen.random_instance(9, 40, seed=3)
    e = oracle.violated_counts(9, cl)
    for x in [0, 1, 77, 255, 300, 511]:
        assert oracle.energy_at(9, cl, x) == e[x]


def test_energy_sum_identity():
    # Each 3-literal clause over distinct variables is violated by exactly
    # 2^(n-3) assignments, so sum_x E(x) = m 2^(n-3).
    import satgen
    n, m = 10, 57
    cl = satgen.random_instance(n, m, seed=11)
    assert int(oracle.violated_counts(n, cl).sum()) == m * (1 << (n - 3))


def test_paper_instance_full_diagonal_and_histogram(paper):
    # Every one of the 64 energies of the worked instance of Sec. 2.2, and their
    # histogram.  A clause with a flipped literal sign, a dropped or duplicated
    # clause, or a transposed bit order changes several entries.
    e = oracle.violated_counts(paper["n"], paper["clauses"])
    assert e.tolist() == paper["diagonal"]
    hist = {str(k): int(v) for k, v in enumerate(np.bincount(e)) if v}
    assert hist == paper["histogram"]
    assert sum(paper["histogram"].values()) == 64
    # each 3-literal clause over distinct variables is violated by 8 of the 64 assignments
    assert int(e.sum()) == 8 * len(paper["clauses"]) == 216


def test_planted_mistakes_change_the_paper_diagonal(paper):
    # The pin above is sensitive: each plausible slip, planted here in a copy of
    # the clause list, moves the diagonal away from the stored one.
    base = [list(c) for c in paper["clauses"]]
    flipped = [list(c) for c in base]
    flipped[5][1] = -flipped[5][1]
    dropped = base[:17] + base[18:]
    reversed_bits = [[(7 - abs(l)) * (1 if l > 0 else -1) for l in c] for c in base]
    for cl in (flipped, dropped, reversed_bits):
        assert oracle.violated_counts(6, cl).tolist() != paper["diagonal"]
