"""Spin-1/2 XXZ Hamiltonians for the oracle (test infrastructure only).

H = J sum_<ij> (Sx_i Sx_j + Sy_i Sy_j + Delta Sz_i Sz_j)      (eq. HeisenbergH)
  = J sum_<ij> (1/2 (S+_i S-_j + S-_i S+_j) + Delta Sz_i Sz_j)

with nearest-neighbour bonds of an open chain.  Site 1 is the most significant
factor of every Kronecker product, and basis state 0 of a site is spin up.
"""
from __future__ import annotations

import numpy as np

SP = np.array([[0.0, 1.0], [0.0, 0.0]])   # S+ |down> = |up>
SM = SP.T.copy()                           # S-
SZ = np.diag([0.5, -0.5])
ID = np.eye(2)


def chain_bonds(L: int):
    """Open-chain nearest-neighbour bonds (i, i+1), 0-based."""
    return [(i, i + 1) for i in range(L - 1)]


def _site_op(op: np.ndarray, i: int, L: int) -> np.ndarray:
    out = np.ones((1, 1))
    for j in range(L):
        out = np.kron(out, op if j == i else ID)
    return out


def dense_xxz(L: int, J: float = 1.0, Delta: float = 1.0, bonds=None) -> np.ndarray:
    """Dense 2^L x 2^L matrix of eq. HeisenbergH (Delta = 0 gives eq. HeisenbergXY)."""
    bonds = chain_bonds(L) if bonds is None else bonds
    n = 2 ** L
    H = np.zeros((n, n))
    ops = {}
    for i in range(L):
        ops[i] = (_site_op(SP, i, L), _site_op(SM, i, L), _site_op(SZ, i, L))
    for (i, j) in bonds:
        spi, smi, szi = ops[i]
        spj, smj, szj = ops[j]
        H += J * (0.5 * (spi @ smj + smi @ spj) + Delta * (szi @ szj))
    return H


def xxz_chain_mpo(L: int, J: float = 1.0, Delta: float = 1.0):
    """Automaton MPO of the open XXZ chain (App. B.1).

    Bond states: 0 = start, 1 = stop, 2/3/4 = "S+ / S- / Sz placed, partner
    pending".  The bulk tensor T[alpha, sigma, sigma', alpha'] carries
    T[start,start] = I, T[stop,stop] = I, T[start,2] = S+, T[start,3] = S-,
    T[start,4] = Sz, T[2,stop] = (J/2) S-, T[3,stop] = (J/2) S+,
    T[4,stop] = J Delta Sz, so D_H = 2 + m_int = 5.  The first site keeps the
    start row, the last site the stop column (the "capping" of App. B.1).

    Returns a list of arrays W[i] with shape (Dl, 2, 2, Dr): index order
    (left bond, row spin sigma, column spin sigma', right bond).
    """
    T = np.zeros((5, 2, 2, 5))
    T[0, :, :, 0] = ID
    T[1, :, :, 1] = ID
    T[0, :, :, 2] = SP
    T[0, :, :, 3] = SM
    T[0, :, :, 4] = SZ
    T[2, :, :, 1] = 0.5 * J * SM
    T[3, :, :, 1] = 0.5 * J * SP
    T[4, :, :, 1] = J * Delta * SZ
    if L == 1:
        return [T[0:1, :, :, 1:2].copy()]
    W = [T[0:1].copy()]
    for _ in range(1, L - 1):
        W.append(T.copy())
    W.append(T[:, :, :, 1:2].copy())
    return W


def identity_mpo(L: int):
    """Bond-dimension-1 MPO of the identity operator."""
    return [ID.reshape(1, 2, 2, 1).copy() for _ in range(L)]


def mpo_to_dense(W) -> np.ndarray:
    """Contract an MPO to its dense 2^L x 2^L matrix (site 1 most significant)."""
    T = W[0]                                  # (1, s, t, r)
    T = T.reshape(2, 2, -1)                   # (S, T, r), S/T = row/col multi-index
    for w in W[1:]:
        S, Tt, r = T.shape
        # (S, T, l) x (l, s, t, r) -> (S, s, T, t, r)
        T = np.einsum("STl,lstr->SsTtr", T, w)
        T = T.reshape(S * 2, Tt * 2, w.shape[3])
    assert T.shape[2] == 1
    return T[:, :, 0]


def dense_bonds(N: int, bonds) -> np.ndarray:
    """Dense 2^N x 2^N matrix of sum over bonds (i, j, J, Delta) of
    J (Sx_i Sx_j + Sy_i Sy_j + Delta Sz_i Sz_j) (eq. HeisenbergH on any graph)."""
    n = 2 ** N
    H = np.zeros((n, n))
    ops = {i: (_site_op(SP, i, N), _site_op(SM, i, N), _site_op(SZ, i, N)) for i in range(N)}
    for (i, j, J, Delta) in bonds:
        spi, smi, szi = ops[i]
        spj, smj, szj = ops[j]
        H += J * (0.5 * (spi @ smj + smi @ spj) + Delta * (szi @ szj))
    return H


def bonds_mpo(N: int, bonds):
    """MPO of the same bond sum by a distance automaton (App. B.1 with longer
    range): besides start and stop, one state per (operator, distance d since
    it was placed) for d = 1 .. R, R the longest bond.  At every site the
    states shift d -> d+1 and those at the distance of a bond that ends here
    close with its coupling.  D = 2 + 3 R: larger than necessary for snakes
    (R = 2W - 1) but direct to check.

    Returns W[i] with shape (Dl, 2, 2, Dr) as xxz_chain_mpo.
    """
    R = max(j - i for (i, j, _, _) in bonds)
    coup = {(i, j): (J, Delta) for (i, j, J, Delta) in bonds}
    D = 2 + 3 * R
    start, stop = 0, 1

    def st(o, d):       # o in 0,1,2 = S+, S-, Sz placed d sites ago
        return 2 + 3 * (d - 1) + o

    first = (SP, SM, SZ)
    W = []
    for s_ in range(N):
        T = np.zeros((D, 2, 2, D))
        T[start, :, :, start] = ID
        T[stop, :, :, stop] = ID
        for o in range(3):
            T[start, :, :, st(o, 1)] = first[o]
            for d in range(1, R):
                T[st(o, d), :, :, st(o, d + 1)] = ID
            for d in range(1, R + 1):
                if (s_ - d, s_) in coup:
                    J, Delta = coup[(s_ - d, s_)]
                    close = (0.5 * J * SM, 0.5 * J * SP, J * Delta * SZ)[o]
                    T[st(o, d), :, :, stop] = close
        if s_ == 0:
            T = T[start:start + 1]
        if s_ == N - 1:
            T = T[:, :, :, stop:stop + 1]
        W.append(T)
    return W


def dense_magnetization(L: int) -> np.ndarray:
    """Dense S^z_tot = sum_i S^z_i (Sec. IV D, Eq. Binder)."""
    return sum(_site_op(SZ, i, L) for i in range(L))


def magnetization_mpo(L: int):
    """S^z_tot as an MPO of bond dimension 2: W = [[I, 0], [S^z, I]] in the
    (done, pending) convention of the chain automaton (row 0 of the first
    site, column 1 of the last)."""
    W = np.zeros((2, 2, 2, 2))
    W[0, :, :, 0] = np.eye(2)
    W[1, :, :, 0] = SZ
    W[1, :, :, 1] = np.eye(2)
    sites = []
    for i in range(L):
        if i == 0:
            sites.append(W[1:2].copy())
        elif i == L - 1:
            sites.append(W[:, :, :, 0:1].copy())
        else:
            sites.append(W.copy())
    return sites


def magnetization_power_mpo(L: int, p: int):
    """(S^z_tot)^p as the exact p-fold MPO product of magnetization_mpo
    (bond 2^p, nothing truncated)."""
    M = magnetization_mpo(L)
    out = [w.copy() for w in M]
    for _ in range(p - 1):
        nxt = []
        for a, b in zip(out, M):
            T = np.einsum("asty,btuz->absuyz", a, b)
            la, lb, _, _, ra, rb = T.shape
            nxt.append(T.reshape(la * lb, 2, 2, ra * rb))
        out = nxt
    return out
