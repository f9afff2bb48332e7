"""Pins of the oracle's MPO-sum compression (App. D.2, Eq. LSESum) and of
the pointwise-Taylor SETTN step (Sec. II C, Eq. Tay) against dense
operators, the matrix exponential and exact diagonalisation."""
import math

import numpy as np
from scipy.linalg import expm

from oracle import exact as ex
from oracle import hamiltonian as hm
from oracle import xtrg as xo


def _random_mpo(rng, dims):
    return [rng.standard_normal((dims[i], 2, 2, dims[i + 1])) for i in range(len(dims) - 1)]


def test_overlap_environments_are_the_frobenius_inner_product():
    rng = np.random.default_rng(1)
    A = _random_mpo(rng, [1, 3, 4, 2, 1])
    B = _random_mpo(rng, [1, 2, 5, 3, 1])
    want = float(np.sum(hm.mpo_to_dense(A) * hm.mpo_to_dense(B)))
    VL = np.ones((1, 1))
    for a, b in zip(A, B):
        VL = xo.overlap_left_update(VL, a, b)
    VR = np.ones((1, 1))
    for a, b in zip(reversed(A), reversed(B)):
        VR = xo.overlap_right_update(VR, a, b)
    assert abs(VL[0, 0] - want) < 1e-12 * abs(want)
    assert abs(VR[0, 0] - want) < 1e-12 * abs(want)


def test_compressed_sum_is_exact_when_the_bond_allows_it():
    """C = 0.7 A - 1.3 B + 0.2 D with D* >= the summed bonds: the variational
    sum reproduces the dense sum (a sign error or a dropped term fails)."""
    rng = np.random.default_rng(2)
    A = _random_mpo(rng, [1, 2, 3, 2, 1])
    B = _random_mpo(rng, [1, 3, 2, 3, 1])
    D = _random_mpo(rng, [1, 2, 2, 2, 1])
    w = [0.7, -1.3, 0.2]
    C = xo.compress_sum([A, B, D], w, A, 64, 3, 1e-15)
    want = sum(x * hm.mpo_to_dense(T) for x, T in zip(w, (A, B, D)))
    got = hm.mpo_to_dense(C)
    assert np.abs(got - want).max() < 1e-11 * np.abs(want).max()


def test_compressed_sum_is_the_best_approximation_at_a_small_bond():
    """At D* below the exact bond, the variational sum is no worse than the
    SVD truncation of the exact direct-sum MPO (both are rank-D* MPOs; the
    variational one minimises the same Frobenius cost)."""
    rng = np.random.default_rng(3)
    A = _random_mpo(rng, [1, 3, 4, 3, 1])
    B = _random_mpo(rng, [1, 3, 4, 3, 1])
    want = hm.mpo_to_dense(A) + hm.mpo_to_dense(B)
    C = xo.compress_sum([A, B], [1.0, 1.0], A, 4, 6, 1e-15)
    direct = xo.right_canonicalize(xo.direct_sum(A, 1.0, B), 1e-15)
    # truncate the direct sum by one left-to-right pass of SVD splits
    T = [w.copy() for w in direct]
    for i in range(len(T) - 1):
        l, _, _, r = T[i].shape
        U, S, Vt = np.linalg.svd(T[i].reshape(l * 4, r), full_matrices=False)
        k = min(4, S.size)
        T[i] = U[:, :k].reshape(l, 2, 2, k)
        T[i + 1] = np.tensordot(S[:k, None] * Vt[:k], T[i + 1], axes=([1], [0]))
    err_var = np.linalg.norm(hm.mpo_to_dense(C) - want)
    err_svd = np.linalg.norm(hm.mpo_to_dense(T) - want)
    assert err_var <= err_svd * (1 + 1e-9)


def test_taylor_step_reproduces_the_matrix_exponential():
    """rho(tau) from the series init, then steps of dtau = tau (a doubling) and
    dtau = 0.3 tau (off the grid): e^{lnc} rho equals expm(-(tau+dtau) H)
    within the Taylor remainder (dtau ||H||)^{Nc+1}/(Nc+1)!."""
    L = 6
    H = hm.xxz_chain_mpo(L, 1.0, 0.8)
    Hd = hm.dense_xxz(L, 1.0, 0.8)
    hn = np.abs(np.linalg.eigvalsh(Hd)).max()
    tau = 0.05
    rho, lnc = xo.init_rho(H, tau, 8, 256, 2, 1e-15)
    for frac in (1.0, 0.3):
        dtau = frac * tau
        order = 8
        r2, lnc2 = xo.settn_step(H, rho, lnc, dtau, order, 256, 2, 1e-15)
        got = math.exp(lnc2) * hm.mpo_to_dense(r2)
        want = expm(-(tau + dtau) * Hd)
        bound = (dtau * hn) ** (order + 1) / math.factorial(order + 1) * np.abs(want).max() * 10
        assert np.abs(got - want).max() <= max(bound, 1e-13 * np.abs(want).max())


def test_settn_run_matches_exact_diagonalisation():
    """SETTN along tau_n = 2^n tau0 (Eq. Tay with dtau = tau_n) on a 5-site
    chain, untruncated: f, u and c_V within 1e-10 of ED up to beta = 1."""
    L = 5
    H = hm.xxz_chain_mpo(L, 1.0, 1.0)
    E = ex.ed_spectrum(hm.dense_xxz(L, 1.0, 1.0))
    rows = xo.run_settn(H, 2.0 ** -6, 6, 64, 2, 6, 16, 1e-15)
    assert abs(rows[-1]["beta"] - 1.0) < 1e-15
    for r in rows:
        e = ex.ed_thermo(E, r["beta"], L)
        assert abs(r["f"] - e["f"]) < 1e-10, (r["beta"], r["f"], e["f"])
        assert abs(r["u"] - e["u"]) < 1e-10
        assert abs(r["c"] - e["c"]) < 1e-9
