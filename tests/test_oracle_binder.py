"""Pins of the Binder-ratio machinery of the oracle (Sec. IV D, Eq. Binder):
the magnetisation MPOs against dense operators, the infinite-temperature
closed form, and XTRG against exact diagonalisation."""
import numpy as np

from oracle import exact as ex
from oracle import hamiltonian as hm
from oracle import xtrg as xo


def test_magnetization_power_mpos_are_the_dense_powers():
    for L in (2, 3, 5):
        M = hm.dense_magnetization(L)
        assert np.abs(hm.mpo_to_dense(hm.magnetization_mpo(L)) - M).max() < 1e-15
        for p in (2, 4):
            want = np.linalg.matrix_power(M, p)
            got = hm.mpo_to_dense(hm.magnetization_power_mpo(L, p))
            assert np.abs(got - want).max() < 1e-13 * max(1.0, np.abs(want).max())


def test_binder_ratio_at_infinite_temperature():
    """rho = identity: independent spins +-1/2 give <M^2> = N/4,
    <M^4> = (3N^2 - 2N)/16, U_4 = N/(3N - 2)."""
    for L in (2, 4, 7):
        rho = hm.identity_mpo(L)
        M2, M4 = hm.magnetization_power_mpo(L, 2), hm.magnetization_power_mpo(L, 4)
        assert abs(xo.expectation(M2, rho) - L / 4) < 1e-13
        assert abs(xo.expectation(M4, rho) - (3 * L * L - 2 * L) / 16) < 1e-12
        assert abs(xo.binder_ratio(M2, M4, rho) - L / (3 * L - 2)) < 1e-13


def test_binder_ratio_of_xtrg_matches_ed():
    L, D = 6, 0.5
    H = hm.xxz_chain_mpo(L, 1.0, D)
    Hd = hm.dense_xxz(L, 1.0, D)
    Md = hm.dense_magnetization(L)
    M2, M4 = hm.magnetization_power_mpo(L, 2), hm.magnetization_power_mpo(L, 4)
    # order-8 series init: its remainder (tau0 ||H||)^9/9! is far below the bar
    rows, states = xo.run_xtrg(H, 2.0 ** -6, 8, 64, 2, 8, 1e-15, keep_states=True)
    for r, (rho, lnc) in zip(rows, states):
        u4 = xo.binder_ratio(M2, M4, rho)
        assert abs(u4 - ex.ed_binder(Hd, Md, r["beta"])) < 1e-10, r["beta"]
