"""The first-order second CholeskyQR pass, checked on the CPU in FP64.

The truncation of the tensor-core path orthonormalises its subspace basis by
scaled CholeskyQR and replaces the second pass, when the first pass left a
basis U1 with U1^T U1 = I + E and max|E| small, by U2 = U1 (I - Phi(E)^T),
Phi(E) = strictly lower part of E plus half its diagonal.  The claim is that
U2^T U2 = I + O(E^2) (the Cholesky factor of I + E is I + Phi(E) + O(E^2)).
This test checks the algebra the kernel relies on, independently of the
kernel: the defect after the correction shrinks quadratically with E (its
second-order terms are sums of k products, so in the max norm it stays below
3 k max|E|^2 and, for these bases, near 4 max|E|^2), and the spanned subspace
is unchanged.
"""
import numpy as np
import pytest


def phi(E):
    return np.tril(E, -1) + 0.5 * np.diag(np.diag(E))


@pytest.mark.parametrize("eps", [1e-2, 3e-3, 1e-3, 3e-4])
def test_first_order_pass_has_quadratic_defect(eps):
    rng = np.random.default_rng(7)
    rows, k = 400, 48
    Q, _ = np.linalg.qr(rng.standard_normal((rows, k)))
    # a nearly orthonormal basis: U1 = Q (I + eps S), S random
    U1 = Q @ (np.eye(k) + eps * rng.standard_normal((k, k)) / np.sqrt(k))
    E = U1.T @ U1 - np.eye(k)
    U2 = U1 @ (np.eye(k) - phi(E).T)
    d1 = np.abs(E).max()
    d2 = np.abs(U2.T @ U2 - np.eye(k)).max()
    assert d2 <= 3.0 * k * d1 ** 2 + 1e-14, (eps, d1, d2)
    assert d2 <= 5.0 * d1 ** 2, (eps, d1, d2)
    assert d2 < 0.05 * d1
    # same column space: the projector onto U2's span equals Q's
    P2 = U2 @ np.linalg.solve(U2.T @ U2, U2.T)
    assert np.abs(P2 - Q @ Q.T).max() < 1e-12


def test_cholesky_of_identity_plus_e_to_first_order():
    """chol(I + E) = I + Phi(E) + O(E^2) for symmetric E."""
    rng = np.random.default_rng(3)
    k = 32
    for eps in (1e-2, 1e-3, 1e-4):
        S = rng.standard_normal((k, k))
        E = eps * (S + S.T) / np.sqrt(k)
        L = np.linalg.cholesky(np.eye(k) + E)
        err = np.abs(L - np.eye(k) - phi(E)).max()
        assert err <= 2.0 * np.abs(E).max() ** 2, (eps, err)


def test_dead_columns_stay_zero():
    """A zero column of U1 (a dropped, numerically dependent column) stays
    zero and does not disturb the others when its row and column of B are
    set as the kernel sets them (B row e_j, zeros elsewhere)."""
    rng = np.random.default_rng(5)
    rows, k, dead = 200, 16, 5
    Q, _ = np.linalg.qr(rng.standard_normal((rows, k)))
    U1 = Q @ (np.eye(k) + 1e-4 * rng.standard_normal((k, k)))
    U1[:, dead] = 0.0
    G = U1.T @ U1
    live = np.diag(G) >= 0.5
    B = np.zeros((k, k))
    for n in range(k):
        for c in range(k):
            if not live[n]:
                B[n, c] = 1.0 if n == c else 0.0
            elif live[c]:
                E = G[n, c] - (1.0 if n == c else 0.0)
                B[n, c] = 1.0 - 0.5 * E if n == c else (-E if n > c else 0.0)
    U2 = U1 @ B.T
    assert np.all(U2[:, dead] == 0.0)
    Gl = (U2.T @ U2)[np.ix_(live, live)]
    assert np.abs(Gl - np.eye(live.sum())).max() < 1e-5
