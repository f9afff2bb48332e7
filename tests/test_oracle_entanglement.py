"""MPO entanglement S_E per bond (Sec. IV, Eq. purif) against its plain
definition: the operator Schmidt decomposition of the dense operator across
the bond, rows (s_1 t_1 ... s_i t_i) and columns (s_{i+1} t_{i+1} ...)."""
import numpy as np
import scipy.linalg as sla

from oracle import exact as ex
from oracle import hamiltonian as oh
from oracle import xtrg as ox


def dense_operator_entropies(R, L):
    """S_E of a dense 2^L x 2^L operator at each of the L-1 bonds."""
    T = R.reshape([2] * (2 * L))               # s_1..s_L, t_1..t_L
    perm = [k for i in range(L) for k in (i, L + i)]
    T = T.transpose(perm)                      # s_1 t_1 s_2 t_2 ...
    out = []
    for i in range(1, L):
        S = np.linalg.svd(T.reshape(4 ** i, -1), compute_uv=False)
        p = S ** 2 / np.sum(S ** 2)
        p = p[p > 1e-300]
        out.append(float(-np.sum(p * np.log(p))))
    return out


def test_random_mpo_matches_dense_definition():
    rng = np.random.default_rng(11)
    dims = [1, 3, 5, 4, 2, 1]
    W = [rng.standard_normal((dims[i], 2, 2, dims[i + 1])) for i in range(5)]
    got = ox.mpo_entanglement(W)
    want = dense_operator_entropies(oh.mpo_to_dense(W), 5)
    assert np.allclose(got, want, atol=1e-12)


def test_product_operators_have_zero_entropy():
    assert np.allclose(ox.mpo_entanglement(oh.identity_mpo(6)), 0.0, atol=1e-14)
    rng = np.random.default_rng(2)
    W = [rng.standard_normal((1, 2, 2, 1)) for _ in range(4)]
    assert np.allclose(ox.mpo_entanglement(W), 0.0, atol=1e-14)


def test_thermal_mpo_matches_dense_exponential():
    L, beta = 6, 0.5
    H = oh.xxz_chain_mpo(L)
    rows, states = ox.run_xtrg(H, 2.0 ** -8, 4, 64, 2, 7, 1e-15, keep_states=True)
    rho, _ = states[-1]
    assert abs(rows[-1]["beta"] - beta) < 1e-15
    got = ox.mpo_entanglement(rho)
    want = dense_operator_entropies(sla.expm(-beta * oh.dense_xxz(L)), L)
    assert np.allclose(got, want, atol=1e-9)


def test_high_temperature_entropy_is_second_order_in_tau():
    """rho = I - tau H: singular values [1, alpha tau] at every bond, so S_E
    grows as tau^2 ln(1/tau) at small tau (Sec. IV)."""
    L = 5
    Hd = oh.dense_xxz(L)
    s1 = dense_operator_entropies(np.eye(2 ** L) - 1e-3 * Hd, L)
    s2 = dense_operator_entropies(np.eye(2 ** L) - 2e-3 * Hd, L)
    for a, b in zip(s1, s2):
        # tau^2 ln(1/tau) scaling: doubling tau multiplies S_E by 4 (1 - ln2/ln(1/tau) ...)
        assert 3.0 < b / a < 4.0
