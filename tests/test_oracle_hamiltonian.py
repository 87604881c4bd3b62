"""Pins for the oracle's Hamiltonians and Walsh-Hadamard transform (Eq. (1), Sec. 2.1)."""

from math import comb

import numpy as np
import pytest
import scipy.linalg

import oracle
from oracle.evolve import popcounts


@pytest.mark.parametrize("n", [1, 2, 3, 5])
def test_hb_spectrum_is_binomial(n):
    # sum_i (I - X_i)/2 has eigenvalue p with multiplicity C(n, p).
    lam = np.linalg.eigvalsh(oracle.hb_dense(n))
    vals, counts = np.unique(np.round(lam, 9), return_counts=True)
    assert vals.tolist() == list(range(n + 1))
    assert counts.tolist() == [comb(n, p) for p in range(n + 1)]


@pytest.mark.parametrize("n", [1, 3, 6])
def test_uniform_state_is_hb_ground_state(n):
    # Sec. 2.1: the initial ground state is the uniform superposition.
    psi = oracle.uniform_state(n)
    assert np.allclose(oracle.hb_dense(n) @ psi, 0.0, atol=1e-13)
    assert abs(oracle.norm(psi) - 1.0) < 1e-14


@pytest.mark.parametrize("n", [1, 2, 4, 7, 10])
def test_wht_matches_sylvester_hadamard(n):
    rng = np.random.default_rng(n)
    v = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    ref = scipy.linalg.hadamard(1 << n) @ v / 2 ** (n / 2)
    assert np.allclose(oracle.wht_normalized(v), ref, atol=1e-12)


@pytest.mark.parametrize("n", [3, 8])
def test_wht_is_an_involution_and_maps_e0_to_uniform(n):
    rng = np.random.default_rng(5)
    v = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    assert np.allclose(oracle.wht_normalized(oracle.wht_normalized(v)), v, atol=1e-12)
    e0 = np.zeros(1 << n, dtype=complex)
    e0[0] = 1
    assert np.allclose(oracle.wht_normalized(e0), oracle.uniform_state(n), atol=1e-14)


@pytest.mark.parametrize("n", [2, 4, 6])
def test_hb_is_popcount_in_hadamard_basis(n):
    # H_B = W diag(popcount) W: the identity the Strang split relies on.
    dim = 1 << n
    w = scipy.linalg.hadamard(dim) / 2 ** (n / 2)
    lhs = w @ np.diag(popcounts(n).astype(float)) @ w
    assert np.allclose(lhs, oracle.hb_dense(n), atol=1e-12)


def test_sigma_x_acts_on_bit_i_minus_1():
    n = 3
    e = np.zeros(8, dtype=complex)
    e[0b001] = 1
    assert np.flatnonzero(oracle.sigma_x_dense(n, 1) @ e).tolist() == [0b000]
    assert np.flatnonzero(oracle.sigma_x_dense(n, 3) @ e).tolist() == [0b101]


def test_h_dense_interpolates():
    cl = [[1, -2, 3], [2, 3, -4]]
    n = 4
    hb, hp = oracle.hb_dense(n), oracle.hp_dense(n, cl)
    assert np.allclose(oracle.h_dense(n, cl, 0.0), hb)
    assert np.allclose(oracle.h_dense(n, cl, 1.0), hp)
    assert np.allclose(oracle.h_dense(n, cl, 0.3), 0.7 * hb + 0.3 * hp)
    assert np.allclose(np.diag(hp).real, oracle.violated_counts(n, cl))
