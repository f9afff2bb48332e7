"""Hamiltonian MPOs for the engine (host, FP64).

A finite-state-automaton construction (App. B.1 of arXiv:1801.00142): the
automaton starts in a "nothing placed yet" state, places the first operator of
a two-body term and carries it along the chain in a "pending" state (one state
per term still open across a bond), and ends in an "all done" state once the
partner operator is placed.  For nearest-neighbour XXZ chains the bond space
holds the two terminal states plus one pending state per operator S+, S-, Sz,
so D_H = 5.  Bond states here are ordered [done, pending..., ready]; the first
site keeps the "ready" row and the last site the "done" column.
"""
from __future__ import annotations

import math

import numpy as np

_I = np.eye(2)
_SP = np.array([[0.0, 1.0], [0.0, 0.0]])
_SM = np.array([[0.0, 0.0], [1.0, 0.0]])
_SZ = np.array([[0.5, 0.0], [0.0, -0.5]])


def xxz_chain(L: int, J: float = 1.0, Delta: float = 1.0):
    """Open XXZ chain H = J sum_i (Sx Sx + Sy Sy + Delta Sz Sz) as an MPO.

    Returns (bond_dims, sites) with sites[i] of shape (Dl, 2, 2, Dr),
    sites[i][l, s, t, r] = coefficient of |s><t|.
    """
    if L < 2:
        raise ValueError("need L >= 2")
    # (first operator, second operator, coupling) of each nearest-neighbour term
    terms = [(_SP, _SM, 0.5 * J), (_SM, _SP, 0.5 * J), (_SZ, _SZ, J * Delta)]
    D = len(terms) + 2
    done, ready = 0, D - 1
    bulk = np.zeros((D, 2, 2, D))
    bulk[done, :, :, done] = _I
    bulk[ready, :, :, ready] = _I
    for p, (first, second, g) in enumerate(terms):
        bulk[ready, :, :, 1 + p] = first          # place the first operator
        bulk[1 + p, :, :, done] = g * second      # close it on the next site
    sites = [bulk[ready:ready + 1].copy()]
    sites += [bulk.copy() for _ in range(L - 2)]
    sites.append(bulk[:, :, :, done:done + 1].copy())
    dims = [1] + [D] * (L - 1) + [1]
    return dims, sites


def xxz_bonds_mpo(N: int, bonds):
    """MPO of H = sum over bonds (i, j, J, Delta), i < j, of
    J (Sx_i Sx_j + Sy_i Sy_j + Delta Sz_i Sz_j), for two-body couplings of any
    range (the snake-mapped 2D lattices of Sec. I).

    The automaton keeps, across each cut between sites c and c+1, one pending
    state per (left site l with a bond reaching past the cut, operator of l):
    the bond space at cut c is [done, (l, S+), (l, S-), (l, Sz) for each such
    l, ready], so D = 2 + 3 |open sites|, which is 5 for a chain and 3W + 2
    for a width-W snake with open boundaries.  At site c+1 a pending state
    either continues (identity) or closes with the partner operator and its
    coupling, or both when l has bonds on both sides of c+1.

    Returns (bond_dims, sites) like xxz_chain.
    """
    if N < 2:
        raise ValueError("need N >= 2")
    terms = {}
    for (i, j, J, Delta) in bonds:
        if not (0 <= i < j < N):
            raise ValueError(f"bad bond {(i, j)}")
        terms[(i, j)] = (float(J), float(Delta))
    last = {}          # last partner of every left site
    for (i, j) in terms:
        last[i] = max(last.get(i, -1), j)
    # open[c]: left sites with a bond crossing the cut after site c
    opened = [sorted(l for l, r in last.items() if l <= c < r) for c in range(N - 1)]
    partner = {"+": _SM, "-": _SP, "z": _SZ}
    first = {"+": _SP, "-": _SM, "z": _SZ}
    ops = ("+", "-", "z")

    def states(c):
        """index map of the bond space at cut c"""
        m = {"done": 0}
        for l in opened[c]:
            for o in ops:
                m[(l, o)] = len(m)
        m["ready"] = len(m)
        return m

    cuts = [states(c) for c in range(N - 1)]
    sites = []
    for s_ in range(N):
        left = cuts[s_ - 1] if s_ > 0 else {"ready": 0}
        right = cuts[s_] if s_ < N - 1 else {"done": 0}
        Wt = np.zeros((len(left), 2, 2, len(right)))
        if "done" in left and "done" in right:
            Wt[left["done"], :, :, right["done"]] = _I
        if "ready" in left and "ready" in right:
            Wt[left["ready"], :, :, right["ready"]] = _I
        for o in ops:
            if "ready" in left and (s_, o) in right:          # place the first operator
                Wt[left["ready"], :, :, right[(s_, o)]] = first[o]
        for key, a in left.items():
            if not isinstance(key, tuple):
                continue
            l, o = key
            if key in right:                                  # carry it past this site
                Wt[a, :, :, right[key]] = _I
            if (l, s_) in terms and "done" in right:           # close it here
                J, Delta = terms[(l, s_)]
                g = J * Delta if o == "z" else 0.5 * J
                Wt[a, :, :, right["done"]] += g * partner[o]
        sites.append(Wt)
    dims = [1] + [len(c) for c in cuts] + [1]
    return dims, sites


def magnetization_power(L: int, p: int):
    """MPO of (S^z_tot)^p, S^z_tot = sum_i S^z_i, with bond dimension p + 1
    (the D = 3 and D = 5 forms of p = 2 and 4 that the Binder ratio of
    Sec. IV D, Eq. Binder, needs).  Multinomial expansion: the bond state k
    counts the power collected so far; site tensor W[k][k'] = (S^z)^(k'-k) /
    (k'-k)! for k' >= k, the first site starts at k = 0 and carries the
    factor p!, the last ends at k' = p.  Returns (bond_dims, sites)."""
    if L < 2 or p < 1:
        raise ValueError("need L >= 2 and p >= 1")
    W = np.zeros((p + 1, 2, 2, p + 1))
    for k in range(p + 1):
        for k2 in range(k, p + 1):
            W[k, :, :, k2] = np.linalg.matrix_power(_SZ, k2 - k) / math.factorial(k2 - k)
    sites = []
    for i in range(L):
        w = W
        if i == 0:
            w = math.factorial(p) * W[0:1]
        if i == L - 1:
            w = w[:, :, :, p:p + 1]
        sites.append(np.ascontiguousarray(w))
    dims = [1] + [p + 1] * (L - 1) + [1]
    return dims, sites
