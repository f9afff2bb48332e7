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
