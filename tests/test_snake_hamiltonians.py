"""Snake-mapped 2D lattices (Sec. I: a width-W lattice as a chain with bonds up
to distance 2W - 1, whose full MPO needs D_H = 3W + 2 states with open
boundaries; App. B for the automaton).  Pins: closed-form spectra of small
clusters, the Tr H / Tr H^2 moments, MPO -> dense equality for the product's
minimal automaton and the oracle's independent distance automaton, and the
oracle's XTRG on a snake against exact diagonalisation."""
import numpy as np
import pytest

import workloads as wl
from oracle import exact as ex
from oracle import hamiltonian as oh
from oracle import xtrg as ox
from paper_1801_00142_gb300.hamiltonians import xxz_bonds_mpo, xxz_chain


def _neighbours_on_lattice(W, Lx, i, j, periodic_y=False):
    pos = {wl.snake_index(x, y, W): (x, y) for x in range(Lx) for y in range(W)}
    (x1, y1), (x2, y2) = pos[i], pos[j]
    dy = abs(y1 - y2)
    if periodic_y:
        dy = min(dy, W - dy)
    return abs(x1 - x2) + dy == 1 or (periodic_y and abs(x1 - x2) == 1 and dy == 1)


def test_square_snake_geometry():
    for W, Lx in [(2, 3), (3, 4), (4, 2)]:
        b = wl.square_snake_bonds(W, Lx)
        assert len(b) == W * (Lx - 1) + Lx * (W - 1)
        assert len({(i, j) for i, j, _, _ in b}) == len(b)
        # the path visits neighbours: (i, i+1) is always a bond
        assert all((i, i + 1, 1.0, 1.0) in b for i in range(W * Lx - 1))
        # the longest bond has range 2W - 1 (Sec. I)
        assert max(j - i for i, j, _, _ in b) == 2 * W - 1
        assert all(_neighbours_on_lattice(W, Lx, i, j) for i, j, _, _ in b)


def test_triangular_yc_geometry():
    W, Lx = 4, 3
    b = wl.triangular_yc_bonds(W, Lx)
    # per column a ring of W bonds; between columns 2W bonds
    assert len(b) == W * Lx + 2 * W * (Lx - 1)
    deg = np.zeros(W * Lx, int)
    for i, j, _, _ in b:
        deg[i] += 1
        deg[j] += 1
    # bulk columns have coordination 6 (triangular lattice), edge columns 4
    pos = {wl.snake_index(x, y, W): x for x in range(Lx) for y in range(W)}
    for s, d in enumerate(deg):
        assert d == (6 if 0 < pos[s] < Lx - 1 else 4)


def test_closed_form_clusters():
    # 2 x 2 open square = 4-site Heisenberg ring: E0 = -2J
    H = oh.dense_bonds(4, wl.square_snake_bonds(2, 2))
    assert abs(np.linalg.eigvalsh(H)[0] + 2.0) < 1e-12
    # a single YC column of width 3 is a triangle: H = (J/2)(S_tot^2 - 9/4),
    # levels -3/4 (two doublets) and +3/4 (quartet)
    E = np.linalg.eigvalsh(oh.dense_bonds(3, wl.triangular_yc_bonds(3, 1)))
    assert np.allclose(E, [-0.75] * 4 + [0.75] * 4, atol=1e-12)


def test_moments_of_bond_sums():
    rng = np.random.default_rng(7)
    b = [(i, j, float(rng.uniform(0.5, 1.5)), float(rng.uniform(0, 1.5)))
         for i, j, _, _ in wl.square_snake_bonds(2, 3)]
    H = oh.dense_bonds(6, b)
    assert abs(np.trace(H)) < 1e-12
    want = sum(J * J * (2 + D * D) / 16 for _, _, J, D in b)
    assert abs(np.trace(H @ H) / 2 ** 6 - want) < 1e-12


@pytest.mark.parametrize("lattice", [("sq", 2, 3), ("sq", 3, 3), ("sq", 2, 5), ("tri", 3, 3)])
def test_mpo_builders_match_dense(lattice):
    kind, W, Lx = lattice
    rng = np.random.default_rng(3)
    gen = wl.square_snake_bonds if kind == "sq" else wl.triangular_yc_bonds
    b = [(i, j, float(rng.uniform(0.5, 1.5)), float(rng.uniform(0, 1.5)))
         for i, j, _, _ in gen(W, Lx)]
    N = W * Lx
    Hd = oh.dense_bonds(N, b)
    dims, sites = xxz_bonds_mpo(N, b)
    assert np.abs(oh.mpo_to_dense(sites) - Hd).max() < 1e-12
    assert np.abs(oh.mpo_to_dense(oh.bonds_mpo(N, b)) - Hd).max() < 1e-12
    assert dims[0] == dims[-1] == 1
    assert all(s.shape == (dims[i], 2, 2, dims[i + 1]) for i, s in enumerate(sites))
    if kind == "sq":
        # D_H = 3W + 2 for the open square snake (Sec. I)
        assert max(dims) == 3 * W + 2


def test_bonds_mpo_of_a_chain_is_the_chain_automaton():
    d1, s1 = xxz_chain(7, 1.0, 0.6)
    d2, s2 = xxz_bonds_mpo(7, wl.chain_bonds(7, 1.0, 0.6))
    assert d1 == d2
    assert np.abs(oh.mpo_to_dense(s1) - oh.mpo_to_dense(s2)).max() < 1e-12


def test_oracle_xtrg_on_square_snake_matches_ed():
    W, Lx = 2, 3
    b = wl.square_snake_bonds(W, Lx)
    N = W * Lx
    H = oh.bonds_mpo(N, b)
    E = ex.ed_spectrum(oh.dense_bonds(N, b))
    # tau0 small enough that the 4th-order series error (tau0 ||H||)^5 / 5!
    # stays below 1e-10 after 12 doublings (||H|| ~ 5 for 7 bonds)
    rows = ox.run_xtrg(H, 2.0 ** -10, 4, 64, 2, 12, 1e-15)
    for r in rows:
        ref = ex.ed_thermo(E, r["beta"], N)
        assert abs(r["lnZ"] - ref["lnZ"]) <= 1e-10 * max(1.0, abs(ref["lnZ"]))
        assert abs(r["u"] - ref["u"]) <= 1e-9


def test_golden_snake_rows_match_ed():
    """The stored oracle rows of the untruncated snake cases equal exact
    diagonalisation (pins the golden files the GPU parity tests read)."""
    import json
    import os
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    for w in wl.small_lattice_cases():
        with open(os.path.join(here, f"oracle_{w.name}.json")) as f:
            gd = json.load(f)
        E = ex.ed_spectrum(oh.dense_bonds(w.N, w.bonds()))
        for r in gd["rows"]:
            ref = ex.ed_thermo(E, r["beta"], w.N)
            if gd["truncated"]:
                # truncation discards weight of the compressed products: for this
                # case ln Z stays at or below the exact value at every beta
                assert r["lnZ"] <= ref["lnZ"] + 1e-9
            else:
                assert abs(r["lnZ"] - ref["lnZ"]) <= 1e-10 * max(1.0, abs(ref["lnZ"]))
                assert abs(r["u"] - ref["u"]) <= 1e-9
