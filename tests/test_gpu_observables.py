"""GPU parity of the observables beyond f, u, c_V: the Binder ratio through
xtrg_expectation (Sec. IV D, Eq. Binder) and the cross products
rho_{n,n'} = rho_a rho_b through xtrg_cross_product (Sec. II B, after
Eq. zshift), against the oracle on the same states and exact
diagonalisation (untruncated chains, FP64 path)."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng_cls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_00142_gb300.build import build
    build()
    from paper_1801_00142_gb300.engine import XTRG
    return XTRG


def test_binder_ratio_matches_oracle_and_ed(eng_cls):
    from oracle import exact as ex
    from oracle import hamiltonian as oh
    from oracle import xtrg as ox
    L, D = 6, 0.5
    Hd = oh.dense_xxz(L, 1.0, D)
    Md = oh.dense_magnetization(L)
    M2, M4 = oh.magnetization_power_mpo(L, 2), oh.magnetization_power_mpo(L, 4)
    eng = eng_cls.xxz(L, 1.0, D, tau0=2.0 ** -6, dstar=64, sweeps=2, order=8)
    eng.init()
    for n in range(9):
        if n:
            eng.double()
        o = eng.observables()
        u4 = eng.binder_ratio()
        sites, lnc, beta = eng.get_state()
        ref = ox.binder_ratio(M2, M4, sites)
        assert abs(u4 - ref) <= 1e-12, (beta, u4, ref)
        assert abs(u4 - ex.ed_binder(Hd, Md, beta)) <= 1e-9, (beta, u4)
        # <H> through the generic expectation is the energy of the observables
        from paper_1801_00142_gb300.hamiltonians import xxz_chain
        assert abs(eng.expectation(*xxz_chain(L, 1.0, D)) - L * o["u"]) <= 1e-11 * L


def test_cross_products_give_intermediate_betas(eng_cls):
    """rho(tau_a) rho(tau_b) from two checkpoints is rho(tau_a + tau_b): the
    3/4 and 3/2 (in units of the grid) points between doublings equal ED,
    and the oracle's compressed product of the same two states."""
    from oracle import exact as ex
    from oracle import hamiltonian as oh
    from oracle import xtrg as ox
    L, D = 6, 1.0
    E = ex.ed_spectrum(oh.dense_xxz(L, 1.0, D))
    eng = eng_cls.xxz(L, 1.0, D, tau0=2.0 ** -4, dstar=64, sweeps=2, order=8)
    eng.init()
    ck, states = [], []
    for n in range(4):
        if n:
            eng.double()
        ck.append(eng.checkpoint())
        states.append(eng.get_state())
    for a, b in ((2, 1), (3, 2), (3, 0)):
        eng.cross_product(ck[a], ck[b])
        g = eng.observables()
        want_beta = states[a][2] + states[b][2]
        assert abs(g["beta"] - want_beta) < 1e-14 * want_beta
        e = ex.ed_thermo(E, want_beta, L)
        assert abs(g["lnZ"] - e["lnZ"]) <= 1e-9 * abs(e["lnZ"]), (a, b, g["lnZ"], e["lnZ"])
        assert abs(g["u"] - e["u"]) <= 1e-9
        ra, la, _ = states[a]
        rb, lb, _ = states[b]
        C = ox.compress_product(ra, rb, ra, 64, 2, 1e-15)
        C, lns = ox.normalize_center(C)
        o = ox.observables(oh.xxz_chain_mpo(L, 1.0, D), C, la + lb + lns, want_beta, L)
        assert abs(g["lnZ"] - o["lnZ"]) <= 1e-11 * abs(o["lnZ"])
        assert math.isfinite(g["c"])
    # the engine continues from a cross product like from any state
    eng.double()
    g = eng.observables()
    assert abs(g["lnZ"] - ex.ed_thermo(E, g["beta"], L)["lnZ"]) <= 1e-9 * abs(g["lnZ"])
