"""Pins of the oracle's spectrum of H(s): closed forms and special cases."""

import math

import numpy as np
import pytest

import oracle
import satgen


@pytest.mark.parametrize("s", [0.0, 0.3, 0.5, 0.9, 1.0])
def test_one_qubit_levels_closed_form(s):
    # clause "x1" is violated by x1 = 0: H = (1-s)(1 - X)/2 + s |0><0|
    # = c I - (a X - b Z)/2 with a = 1-s, b = s, c = (a+b)/2: levels c -/+ sqrt(a^2+b^2)/2
    a, b = 1.0 - s, s
    c, om = 0.5 * (a + b), 0.5 * math.hypot(a, b)
    lam = oracle.eigenvalues(1, [[1]], s)
    assert np.allclose(lam, [c - om, c + om], atol=1e-14)
    # both levels overlap the uniform state unless it is an eigenvector (s = 0)
    lv = oracle.sector_eigenvalues(1, [[1]], s, 2)
    assert len(lv) == (1 if s == 0.0 else 2)
    assert abs(lv[0] - (c - om)) < 1e-14


def test_s_zero_sector_is_the_uniform_state_alone():
    cl = satgen.planted_instance(8, 1)["clauses"]
    lv = oracle.sector_eigenvalues(8, cl, 0.0, 3)
    assert len(lv) == 1 and abs(lv[0]) < 1e-12          # H_B's ground level, energy 0
    lam = oracle.eigenvalues(8, cl, 0.0)
    assert abs(lam[0]) < 1e-12 and abs(lam[1] - 1.0) < 1e-12 and abs(lam[8] - 1.0) < 1e-12  # level 1, multiplicity 8


def test_s_one_levels_are_the_clause_counts():
    cl = satgen.ratio_instance(9, 3, min_solutions=2)["clauses"]
    e = oracle.violated_counts(9, cl)
    lv = oracle.sector_eigenvalues(9, cl, 1.0, 3)
    assert np.allclose(lv, np.unique(e)[:3], atol=1e-12)  # every basis state overlaps the uniform state


def test_planted_instance_gap_closes_in_the_middle():
    cl = satgen.planted_instance(8, 2)["clauses"]
    gaps = [oracle.sector_gap(8, cl, s) for s in np.linspace(0.05, 1.0, 20)]
    assert all(g > 0 for g in gaps)
    assert min(gaps) < gaps[0] and min(gaps) < gaps[-1]


def test_sparse_levels_agree_with_dense():
    cl = satgen.ratio_instance(9, 4, min_solutions=1)["clauses"]
    for s in (0.2, 0.6):
        dense = np.unique(np.round(oracle.eigenvalues(9, cl, s), 9))[:3]
        assert np.allclose(oracle.sparse_levels(9, cl, s, 3), dense, atol=1e-8)
