"""Pins for the oracle's exact references: closed forms and brute force.

Two independent constructions must agree: the dense Kronecker-product
Hamiltonian with ED, the automaton MPO of App. B.1, the free-fermion closed
form of App. F, and the single-bond spectrum.
"""
import numpy as np
import pytest

from oracle import exact as ex
from oracle import hamiltonian as hm


@pytest.mark.parametrize("J,Delta", [(1.0, 1.0), (1.0, 0.0), (0.7, 1.9)])
def test_two_site_spectrum_closed_form(J, Delta):
    E = np.sort(ex.ed_spectrum(hm.dense_xxz(2, J, Delta)))
    ref = np.sort([J * Delta / 4, J * Delta / 4, -J * Delta / 4 + J / 2, -J * Delta / 4 - J / 2])
    assert np.allclose(E, ref, atol=1e-14)
    for beta in (0.1, 1.0, 7.0):
        assert abs(ex.ed_thermo(E, beta, 2)["lnZ"] - ex.two_site_lnZ(beta, J, Delta)) < 1e-13


def test_heisenberg_bond_worked_example():
    # Delta = 1: singlet at -3/4, triplet at +1/4 -> Z = 3 e^{-beta/4} + e^{3 beta/4}
    for beta in (0.5, 2.0, 10.0):
        assert abs(ex.two_site_lnZ(beta, 1.0, 1.0)
                   - np.log(3 * np.exp(-beta / 4) + np.exp(3 * beta / 4))) < 1e-13


@pytest.mark.parametrize("L,Delta", [(3, 1.0), (5, 0.3), (6, 1.5)])
def test_high_temperature_moments(L, Delta):
    H = hm.dense_xxz(L, 1.0, Delta)
    n = 2 ** L
    assert abs(np.trace(H)) < 1e-12
    assert abs(np.trace(H @ H) / n - (L - 1) * (2 + Delta ** 2) / 16) < 1e-12
    # second-order expansion of ln Z at small beta
    E = ex.ed_spectrum(H)
    beta = 1e-3
    assert abs(ex.ed_thermo(E, beta, L)["lnZ"] - ex.high_t_lnZ(L, beta, 1.0, Delta)) < 1e-8


@pytest.mark.parametrize("L", [2, 5, 8])
def test_free_fermion_closed_form_matches_ed(L):
    E = ex.ed_spectrum(hm.dense_xxz(L, 1.0, 0.0))
    for beta in (0.01, 0.3, 2.0, 16.0):
        a = ex.free_fermion_thermo(L, beta)
        b = ex.ed_thermo(E, beta, L)
        for k in ("lnZ", "f", "u", "c", "lnZ2"):
            assert abs(a[k] - b[k]) <= 1e-11 * max(1.0, abs(b[k])), (k, beta, a[k], b[k])


def test_free_fermion_limits():
    L = 64
    assert abs(ex.free_fermion_thermo(L, 1e-9)["lnZ"] - L * np.log(2)) < 1e-8
    # ground state: all negative-energy modes filled
    eps = ex.free_fermion_eps(L)
    beta = 400.0
    assert abs(ex.free_fermion_thermo(L, beta)["u"] - eps[eps < 0].sum() / L) < 1e-6


@pytest.mark.parametrize("L,Delta", [(2, 1.0), (4, 0.0), (6, 1.0), (7, 0.45)])
def test_automaton_mpo_matches_dense(L, Delta):
    W = hm.xxz_chain_mpo(L, 1.0, Delta)
    assert [w.shape[3] for w in W[:-1]] == [5] * (L - 1)
    assert np.abs(hm.mpo_to_dense(W) - hm.dense_xxz(L, 1.0, Delta)).max() < 1e-14


def test_identity_mpo():
    assert np.array_equal(hm.mpo_to_dense(hm.identity_mpo(5)), np.eye(32))
