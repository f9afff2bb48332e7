"""Pins for the oracle's CPU XTRG against exact results.

* each contraction against a dense brute-force evaluation on tiny random MPOs
* the SVD split against the Eckart-Young optimum
* the variational compression of an exactly representable product (D* large)
  against the dense product
* the series initialisation against expm(-tau0 H)
* full runs against ED (XXX and XXZ) and against the free-fermion closed form
  (XY), plus the L = 2 worked example and the beta -> 0 limit
* a planted mistake (a transposed operand) in the oracle makes a pin fail
"""
import numpy as np
import pytest
from scipy.linalg import expm

from oracle import exact as ex
from oracle import hamiltonian as hm
from oracle import xtrg as xo


def rand_mpo(rng, L, D):
    dims = [1] + [min(D, 4 ** min(i, L - i)) for i in range(1, L)] + [1]
    return [rng.standard_normal((dims[i], 2, 2, dims[i + 1])) for i in range(L)]


def dense(W):
    return hm.mpo_to_dense(W)


def test_env_updates_brute_force():
    rng = np.random.default_rng(1)
    L = 4
    A, B, C = rand_mpo(rng, L, 3), rand_mpo(rng, L, 2), rand_mpo(rng, L, 3)
    # <C, A^T B>_F from the left environment chain and the right chain
    V = np.ones((1, 1, 1))
    for i in range(L):
        V = xo.left_env_update(V, A[i], B[i], C[i])
    R = np.ones((1, 1, 1))
    for i in range(L - 1, -1, -1):
        R = xo.right_env_update(R, A[i], B[i], C[i])
    ref = np.sum(dense(C) * (dense(A).T @ dense(B)))
    assert abs(V.item() - ref) < 1e-10 * abs(ref)
    assert abs(R.item() - ref) < 1e-10 * abs(ref)


def test_two_site_overlap_brute_force():
    rng = np.random.default_rng(2)
    L = 4
    A, B = rand_mpo(rng, L, 3), rand_mpo(rng, L, 2)
    C = xo.right_canonicalize(rand_mpo(rng, L, 4), 1e-15)
    # left-orthonormalise site 0 so that sites (1, 2) form the centre
    U, S, Vt = np.linalg.svd(C[0].reshape(4, -1), full_matrices=False)
    C[0] = U.reshape(1, 2, 2, -1)
    VL = xo.left_env_update(np.ones((1, 1, 1)), A[0], B[0], C[0])
    VR = xo.right_env_update(np.ones((1, 1, 1)), A[3], B[3], C[3])
    CE = xo.two_site_overlap(VL, A[1], B[1], A[2], B[2], VR)
    # brute force: <C with sites 1,2 replaced by a unit tensor, A^T B>
    T = dense(A).T @ dense(B)
    c, _, _, _, _, z = CE.shape
    for idx in [(0, 0, 1, 1, 0, 0), (c - 1, 1, 0, 1, 1, z - 1), (1, 1, 1, 0, 0, 2)]:
        E = np.zeros((c, 2, 2, 2, 2, z))
        E[idx] = 1.0
        Ci = E.reshape(c, 2, 2, 4 * z)
        # write the unit tensor as two sites via an identity split
        left = np.eye(c * 4).reshape(c, 2, 2, c * 4)
        right = E.reshape(c * 4, 2, 2, z)
        W = [C[0], left, right, C[3]]
        ref = np.sum(dense(W) * T)
        assert abs(CE[idx] - ref) < 1e-10 * max(1.0, abs(ref))


def test_split_is_eckart_young():
    rng = np.random.default_rng(3)
    CE = rng.standard_normal((3, 2, 2, 2, 2, 5))
    M = CE.reshape(12, 20)
    S = np.linalg.svd(M, compute_uv=False)
    for k in (1, 4, 12):
        for direction in ("right", "left"):
            Ci, Cj, disc, _ = xo.split_two_site(CE, direction, k, 1e-15)
            R = Ci.reshape(12, -1) @ Cj.reshape(Cj.shape[0], -1)
            assert abs(np.linalg.norm(M - R) ** 2 - np.sum(S[k:] ** 2)) < 1e-10
            assert abs(disc - np.sum(S[k:] ** 2) / np.sum(S ** 2)) < 1e-12
            Q = Ci.reshape(12, -1) if direction == "right" else Cj.reshape(Cj.shape[0], -1).T
            assert np.allclose(Q.T @ Q, np.eye(Q.shape[1]), atol=1e-12)


def test_compress_exact_product():
    rng = np.random.default_rng(4)
    L = 5
    A, B = rand_mpo(rng, L, 3), rand_mpo(rng, L, 2)
    st = xo.CompressStats()
    C = xo.compress_product(A, B, xo.exact_product(A, B), 256, 2, 1e-15, st)
    ref = dense(A).T @ dense(B)
    assert np.abs(dense(C) - ref).max() < 1e-11 * np.abs(ref).max()
    assert st.max_discarded < 1e-20
    # right-orthonormal sites 1..L-1
    for w in C[1:]:
        M = w.reshape(w.shape[0], -1)
        assert np.allclose(M @ M.T, np.eye(M.shape[0]), atol=1e-12)


def test_compress_from_poor_guess_converges():
    rng = np.random.default_rng(5)
    L = 6
    A = rand_mpo(rng, L, 2)
    C = xo.compress_product(A, A, hm.identity_mpo(L), 256, 4, 1e-15)
    ref = dense(A).T @ dense(A)
    assert np.abs(dense(C) - ref).max() < 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("L,Delta,tau0,order", [(5, 1.0, 2 ** -6, 4), (6, 0.4, 2 ** -10, 4),
                                                  (6, 1.0, 2 ** -14, 1)])
def test_init_matches_expm(L, Delta, tau0, order):
    H = hm.xxz_chain_mpo(L, 1.0, Delta)
    Hd = hm.dense_xxz(L, 1.0, Delta)
    rho, lnc = xo.init_rho(H, tau0, order, 256, 4, 1e-15)
    R = np.exp(lnc) * dense(rho)
    # the series of Eq. RhoTau truncated at Nc
    S = np.zeros_like(Hd)
    term = np.eye(2 ** L)
    for k in range(order + 1):
        S += term
        term = term @ (-tau0 * Hd) / (k + 1)
    assert np.abs(R - S).max() < 1e-13 * np.abs(S).max()
    # and the series error bound (tau0 ||H||)^{Nc+1}/(Nc+1)! against expm
    nrm = np.abs(np.linalg.eigvalsh(Hd)).max()
    bound = (tau0 * nrm) ** (order + 1) / np.prod(np.arange(1, order + 2)) * 1.01 + 1e-14
    assert np.abs(R - expm(-tau0 * Hd)).max() <= bound * np.abs(S).max()


def _run_vs(rows, ref_fn, tol_f, tol_u, tol_c):
    for r in rows:
        e = ref_fn(r["beta"])
        assert abs(r["f"] - e["f"]) <= tol_f * max(1.0, abs(e["f"])), (r["beta"], r["f"], e["f"])
        assert abs(r["u"] - e["u"]) <= tol_u, (r["beta"], r["u"], e["u"])
        assert abs(r["c"] - e["c"]) <= tol_c, (r["beta"], r["c"], e["c"])


@pytest.mark.parametrize("L,Delta", [(5, 1.0), (6, 0.7)])
def test_xtrg_matches_ed(L, Delta):
    H = hm.xxz_chain_mpo(L, 1.0, Delta)
    E = ex.ed_spectrum(hm.dense_xxz(L, 1.0, Delta))
    rows = xo.run_xtrg(H, 2 ** -8, 4, 256, 4, 11, 1e-15)
    assert abs(rows[-1]["beta"] - 8.0) < 1e-12
    _run_vs(rows, lambda b: ex.ed_thermo(E, b, L), 1e-10, 1e-10, 1e-9)
    for r in rows:
        assert abs(r["lnZ2"] - ex.ed_thermo(E, r["beta"], L)["lnZ2"]) < 1e-8


def test_xtrg_xy_matches_free_fermions():
    L = 6
    H = hm.xxz_chain_mpo(L, 1.0, 0.0)
    rows = xo.run_xtrg(H, 2 ** -9, 4, 256, 4, 12, 1e-15)
    _run_vs(rows, lambda b: ex.free_fermion_thermo(L, b), 1e-10, 1e-10, 1e-9)


def test_xtrg_two_sites_worked_example():
    H = hm.xxz_chain_mpo(2, 1.0, 1.0)
    rows = xo.run_xtrg(H, 2 ** -10, 4, 16, 2, 14, 1e-15)
    for r in rows:
        assert abs(r["lnZ"] - ex.two_site_lnZ(r["beta"])) < 1e-11 * max(1, r["beta"])


def test_high_temperature_limit_and_positivity():
    L = 6
    H = hm.xxz_chain_mpo(L, 1.0, 1.0)
    rows = xo.run_xtrg(H, 2 ** -12, 4, 64, 2, 3, 1e-15)
    for r in rows:
        # next term is O(beta^3 Tr H^3 / 2^N) <= (L-1) beta^3 (3/4)^3 / 6
        assert abs(r["lnZ"] - ex.high_t_lnZ(L, r["beta"])) < (L - 1) * r["beta"] ** 3 * 0.0704 + 1e-13
        assert r["herm"] < 1e-6


def test_truncated_run_is_variational():
    # with a small D* the free energy lies above the exact one
    # (Tr rho_trunc <= Tr rho is not guaranteed, but the Frobenius-optimal
    #  compression of rho^T rho never increases ||.||_F: lnZ2 <= exact)
    L = 8
    H = hm.xxz_chain_mpo(L, 1.0, 1.0)
    E = ex.ed_spectrum(hm.dense_xxz(L, 1.0, 1.0))
    rows = xo.run_xtrg(H, 2 ** -8, 4, 12, 2, 9, 1e-15)
    assert max(r["trunc"] for r in rows[1:]) > 1e-8
    for r in rows:
        assert r["lnZ2"] <= ex.ed_thermo(E, r["beta"], L)["lnZ2"] + 1e-9
    # and still close: truncation error in f below 1e-3 at D* = 12
    assert abs(rows[-1]["f"] - ex.ed_thermo(E, rows[-1]["beta"], L)["f"]) < 1e-3


def test_planted_mistake_is_caught(monkeypatch):
    """A transposed operand in the left half of C_E (s and u exchanged) must
    break the ED pin: the pins are sensitive to that class of mistake."""
    good = xo.left_part

    def bad(VL, A, B):
        return good(VL, A, B).transpose(0, 2, 1, 3, 4)

    monkeypatch.setattr(xo, "left_part", bad)
    L = 4
    H = hm.xxz_chain_mpo(L, 1.0, 0.6)
    E = ex.ed_spectrum(hm.dense_xxz(L, 1.0, 0.6))
    H2 = [h.copy() for h in H]
    H2[1][0, :, :, 2] += 0.3 * hm.SZ     # break the s <-> u symmetry of the input
    rho, lnc = xo.init_rho(H2, 2 ** -4, 4, 256, 4, 1e-15)
    monkeypatch.setattr(xo, "left_part", good)
    rho_good, lnc_good = xo.init_rho(H2, 2 ** -4, 4, 256, 4, 1e-15)
    assert np.abs(np.exp(lnc) * dense(rho) - np.exp(lnc_good) * dense(rho_good)).max() > 1e-6


def test_transfer_traces_match_dense_on_a_nonsymmetric_mpo():
    """The transfer-matrix traces of the oracle against the dense operator of
    a random, non-symmetric MPO (so Tr(R R) differs from ||R||_F^2 and from
    Tr(R^T R)): a contraction of Tr(rho rho) that paired the physical indices
    like the Frobenius norm, or a trace that summed the wrong pair, fails."""
    rng = np.random.default_rng(11)
    dims = [1, 3, 5, 4, 1]
    W = [rng.standard_normal((dims[i], 2, 2, dims[i + 1])) for i in range(4)]
    R = hm.mpo_to_dense(W)
    assert np.abs(R - R.T).max() > 1e-2            # genuinely non-symmetric
    assert abs(xo.trace(W) - np.trace(R)) < 1e-12 * np.abs(R).sum()
    assert abs(xo.frobenius2(W) - np.sum(R * R)) < 1e-12 * np.sum(R * R)
    assert abs(xo.trace_rho_rho(W) - np.trace(R @ R)) < 1e-12 * np.sum(R * R)
    H = hm.xxz_chain_mpo(4, 1.0, 0.6)
    Hd = hm.mpo_to_dense(H)
    assert abs(xo.trace_H_rho(H, W) - np.trace(Hd @ R)) < 1e-12 * np.abs(Hd).sum() * np.abs(R).max()
    assert abs(xo.trace_H2_rho(H, W) - np.trace(Hd @ Hd @ R)) < 1e-11 * np.sum(Hd * Hd) * np.abs(R).max() * 16
    # the Hermiticity defect of observables() is ||R - R^T||_F / ||R||_F
    o = xo.observables(H, W, 0.0, 1.0, 4)
    want = np.linalg.norm(R - R.T) / np.linalg.norm(R)
    assert abs(o["herm"] - want) < 1e-10
    # and it vanishes for a symmetrised MPO (R + R^T as a direct sum)
    WT = [w.transpose(0, 2, 1, 3) for w in W]
    S = xo.direct_sum(W, 1.0, WT)
    assert np.abs(hm.mpo_to_dense(S) - (R + R.T)).max() < 1e-12 * np.abs(R).max() * 8
    assert xo.observables(H, S, 0.0, 1.0, 4)["herm"] < 1e-7
