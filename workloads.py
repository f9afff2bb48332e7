"""Seeded synthetic workloads for the XTRG doubling path.

This module holds only workload *descriptions*: chain lengths, couplings,
initial inverse temperatures, bond-dimension caps, sweep counts, and the seeded
draws of the batched workload.  It contains none of the method's arithmetic
(no MPO construction, no contraction, no thermodynamics), so both the CUDA
path and the FP64 oracle may import it without sharing any computation.

The workloads follow the paper's model systems: spin-1/2 Heisenberg XXZ chains
with open boundaries and J = 1 (Sec. I, eq. HeisenbergH; the XY special case
Delta = 0 is eq. HeisenbergXY), cooled by beta doubling from a small initial
tau0 (Sec. II B), with the series initialisation of Eq. RhoTau (Sec. II C).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import List

import numpy as np


@dataclass(frozen=True)
class ChainWorkload:
    """One XTRG run on an open XXZ chain.

    L            number of sites (N = L for a chain)
    J, Delta     couplings of H = J sum_i (Sx Sx + Sy Sy + Delta Sz Sz)
    tau0         initial inverse temperature of rho(tau0)
    order        series order Nc of Eq. RhoTau (terms k = 0..Nc)
    dstar        bond-dimension cap D* of the compressed MPO
    sweeps       full sweeps (left-to-right then right-to-left) per product
    n_doublings  number of doublings after the initialisation
    init_sweeps  sweeps per product inside the series initialisation
    svd_rel_tol  singular values below svd_rel_tol * sigma_max are numerically zero
    """

    name: str
    L: int
    J: float = 1.0
    Delta: float = 1.0
    tau0: float = 2.0 ** -10
    order: int = 4
    dstar: int = 256
    sweeps: int = 4
    n_doublings: int = 15
    init_sweeps: int = 4
    svd_rel_tol: float = 1e-15

    def with_(self, **kw) -> "ChainWorkload":
        return replace(self, **kw)

    @property
    def betas(self) -> List[float]:
        return [self.tau0 * 2.0 ** n for n in range(self.n_doublings + 1)]


# Untruncated check case: L = 8, D* = 256 = 4^4 = the largest exact bond of an
# 8-site MPO, tau0 = 2^-10, 15 doublings to beta = 32.
CHAIN_L8 = ChainWorkload(name="xxz_L8_D256_fp64", L=8, Delta=1.0,
                         tau0=2.0 ** -10, dstar=256, sweeps=4, n_doublings=15)

# Headline case: L = 64, D* = 256, tau0 = 2^-12, 18 doublings to beta = 64,
# 4 sweeps per doubling; Delta in {0, 1}.
CHAIN_L64_XX = ChainWorkload(name="xx_L64_D256", L=64, Delta=0.0,
                             tau0=2.0 ** -12, dstar=256, sweeps=4, n_doublings=18)
CHAIN_L64_XXX = ChainWorkload(name="xxx_L64_D256", L=64, Delta=1.0,
                              tau0=2.0 ** -12, dstar=256, sweeps=4, n_doublings=18)
# The same schedule on a 32-site XX chain: the FP64 reference of the
# mixed-precision accuracy gate at a length the oracle finishes in hours.
CHAIN_L32_XX = ChainWorkload(name="xx_L32_D256", L=32, Delta=0.0,
                             tau0=2.0 ** -12, dstar=256, sweeps=4, n_doublings=18)


def batched_instances(n: int = 64, seed: int = 180100142, n_grids: int = 8,
                      beta_final: float = 64.0) -> List[ChainWorkload]:
    """Seeded batched workload: n chains with L in {16,24,32,48,64},
    Delta ~ U[0, 1.5], D* in {64,128,256}; each chain is run on n_grids
    interleaved tau0 grids tau0 = 2^-12 * 2^(k/n_grids) (the z-shifts of
    Eq. zshift), doubled until beta >= beta_final."""
    rng = np.random.default_rng(seed)
    Ls = rng.choice([16, 24, 32, 48, 64], size=n)
    Deltas = rng.uniform(0.0, 1.5, size=n)
    Ds = rng.choice([64, 128, 256], size=n)
    out = []
    for i in range(n):
        for k in range(n_grids):
            tau0 = 2.0 ** -12 * 2.0 ** (k / n_grids)
            nd = int(np.ceil(np.log2(beta_final / tau0) - 1e-12))
            out.append(ChainWorkload(name=f"inst{i}_z{k}", L=int(Ls[i]),
                                     Delta=float(Deltas[i]), tau0=tau0,
                                     dstar=int(Ds[i]), sweeps=4, n_doublings=nd))
    return out


def small_cases() -> List[ChainWorkload]:
    """Small parity cases the oracle finishes in seconds; they span several
    bond-dimension regimes (growing, saturated, truncated) and both couplings."""
    return [
        ChainWorkload(name="xxx_L4", L=4, Delta=1.0, tau0=2.0 ** -6, dstar=16, n_doublings=8),
        ChainWorkload(name="xx_L6", L=6, Delta=0.0, tau0=2.0 ** -8, dstar=64, n_doublings=10),
        ChainWorkload(name="xxz_L6_trunc", L=6, Delta=0.7, tau0=2.0 ** -8, dstar=12, n_doublings=10),
        ChainWorkload(name="xxx_L10_trunc", L=10, Delta=1.0, tau0=2.0 ** -8, dstar=24,
                      sweeps=2, n_doublings=10),
    ]


# ------------------------------------------------------------------ lattices
# Two-dimensional lattices mapped to a snake path (Sec. I: a width-W system
# becomes a chain with bonds up to distance 2W - 1).  Site (x, y), x along the
# length, y across the width, has index x*W + y on even columns and
# x*W + (W-1-y) on odd columns, so consecutive sites along the path are
# neighbours.  A bond list is a list of (i, j, J, Delta) with i < j: the
# coupling J (Sx Sx + Sy Sy + Delta Sz Sz) between path sites i and j.  These
# are model descriptions only (no Hamiltonian arithmetic).

def snake_index(x: int, y: int, W: int) -> int:
    return x * W + (y if x % 2 == 0 else W - 1 - y)


def _bond(i: int, j: int, J: float, Delta: float):
    return (min(i, j), max(i, j), float(J), float(Delta))


def chain_bonds(L: int, J: float = 1.0, Delta: float = 1.0):
    """Open chain: nearest-neighbour bonds (i, i+1)."""
    return [(i, i + 1, float(J), float(Delta)) for i in range(L - 1)]


def square_snake_bonds(W: int, Lx: int, J: float = 1.0, Delta: float = 1.0):
    """W x Lx square lattice, open boundaries in both directions."""
    bonds = []
    for x in range(Lx):
        for y in range(W):
            i = snake_index(x, y, W)
            if y + 1 < W:
                bonds.append(_bond(i, snake_index(x, y + 1, W), J, Delta))
            if x + 1 < Lx:
                bonds.append(_bond(i, snake_index(x + 1, y, W), J, Delta))
    return sorted(bonds)


def triangular_yc_bonds(W: int, Lx: int, J: float = 1.0, Delta: float = 1.0):
    """Triangular lattice on a YC cylinder: periodic across the width W (one
    lattice direction wraps the circumference), open along the length Lx.
    Each site (x, y) couples to (x, y+1 mod W), (x+1, y) and (x+1, y-1 mod W)."""
    if W < 3:
        raise ValueError("a YC cylinder needs W >= 3")
    bonds = set()
    for x in range(Lx):
        for y in range(W):
            i = snake_index(x, y, W)
            bonds.add(_bond(i, snake_index(x, (y + 1) % W, W), J, Delta))
            if x + 1 < Lx:
                bonds.add(_bond(i, snake_index(x + 1, y, W), J, Delta))
                bonds.add(_bond(i, snake_index(x + 1, (y - 1) % W, W), J, Delta))
    return sorted(bonds)


@dataclass(frozen=True)
class LatticeWorkload:
    """One XTRG run on a snake-mapped 2D lattice (kind "square": open W x Lx;
    "triangular_yc": YC cylinder of circumference W and length Lx)."""

    name: str
    kind: str
    W: int
    Lx: int
    J: float = 1.0
    Delta: float = 1.0
    tau0: float = 2.0 ** -10
    order: int = 4
    dstar: int = 500
    sweeps: int = 4
    n_doublings: int = 15
    n_grids: int = 1
    svd_rel_tol: float = 1e-15

    @property
    def N(self) -> int:
        return self.W * self.Lx

    def bonds(self):
        gen = square_snake_bonds if self.kind == "square" else triangular_yc_bonds
        return gen(self.W, self.Lx, self.J, self.Delta)


# 6 x 6 open square Heisenberg lattice, tau0 = 2^-10 doubled to beta = 32, D* = 500.
SQUARE_6X6 = LatticeWorkload(name="square_6x6_D500", kind="square", W=6, Lx=6, dstar=500)
# Triangular Heisenberg 6 x 6 YC cylinder and the easy-plane (Delta = 0.5) 8 x 8
# square lattice, D* = 768, 4 interleaved tau0 grids each.
TRIANGULAR_YC6X6 = LatticeWorkload(name="triangular_yc6x6_D768", kind="triangular_yc", W=6, Lx=6,
                                   dstar=768, n_grids=4)
SQUARE_8X8_XXZ = LatticeWorkload(name="square_8x8_xxz_D768", kind="square", W=8, Lx=8,
                                 Delta=0.5, dstar=768, n_grids=4)


def small_lattice_cases() -> List[LatticeWorkload]:
    """Snake-lattice parity cases the oracle finishes in seconds: an
    untruncated and a truncated open square strip and an untruncated
    triangular YC cylinder, tau0 = 2^-10 doubled to beta = 4.  The truncated
    strip takes 6 sweeps per product, enough for the variational compression
    to reach its fixed point, so GPU and CPU agree to their rounding
    sensitivity there too."""
    return [
        LatticeWorkload(name="square_2x3", kind="square", W=2, Lx=3, dstar=64, sweeps=2,
                        n_doublings=12),
        LatticeWorkload(name="square_2x3_trunc", kind="square", W=2, Lx=3, dstar=20, sweeps=6,
                        n_doublings=12),
        LatticeWorkload(name="triangular_yc3x2", kind="triangular_yc", W=3, Lx=2, dstar=64,
                        sweeps=2, n_doublings=12),
    ]
