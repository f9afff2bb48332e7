"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Observables are gauge invariant, so runs are compared per beta on ln Z, f, u,
c_V; states are compared through their dense matrices (small L) or through
bond dimensions and traces.  The FP64 path must agree with the oracle to the
accumulated-rounding level (the oracle itself agrees with ED to ~1e-11), so
the bars are |d lnZ| <= 1e-10 max(1, |lnZ|), |du| <= 1e-10, |dc| <= 1e-9.
"""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def eng_cls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_00142_gb300.build import build
    build()
    from paper_1801_00142_gb300.engine import XTRG
    return XTRG


def golden(name):
    with open(os.path.join(HERE, "golden", f"oracle_{name}.json")) as f:
        return json.load(f)


def compare_rows(gpu, ref, tol_lnz=1e-10, tol_u=1e-10, tol_c=1e-9):
    """Per-beta comparison.  For truncated runs the golden rows carry the
    oracle's own sensitivity (largest change over three 1e-14 perturbations
    of H); the bar is then max(tol, 300 * sensitivity): the GPU's rounding
    differs from the CPU's by more than one such perturbation."""
    assert len(gpu) == len(ref)
    for g, o in zip(gpu, ref):
        sens = o.get("sens", {"lnZ": 0.0, "u": 0.0, "c": 0.0})
        assert abs(g["beta"] - o["beta"]) < 1e-14 * o["beta"]
        bar = max(tol_lnz * max(1.0, abs(o["lnZ"])), 300 * sens["lnZ"])
        assert abs(g["lnZ"] - o["lnZ"]) <= bar, (o["beta"], g["lnZ"], o["lnZ"], bar)
        assert abs(g["u"] - o["u"]) <= max(tol_u, 300 * sens["u"]), (o["beta"], g["u"], o["u"])
        assert abs(g["c"] - o["c"]) <= max(tol_c, 300 * sens["c"]), (o["beta"], g["c"], o["c"])


def bonds_close(a, b, slack=2):
    """Bond dimensions agree up to the singular values that sit at the
    numerical-zero threshold (rel_tol * sigma_max), whose count is decided
    by rounding."""
    return abs(a - b) <= slack


@pytest.mark.parametrize("name", ["xxx_L4", "xx_L6", "xxz_L6_trunc", "xxx_L10_trunc"])
def test_small_cases_match_oracle(eng_cls, name):
    gd = golden(name)
    w = gd["workload"]
    eng = eng_cls.xxz(w["L"], w["J"], w["Delta"], tau0=w["tau0"], dstar=w["dstar"],
                      sweeps=w["sweeps"], order=w["order"], init_sweeps=w["init_sweeps"],
                      svd_rel_tol=w["svd_rel_tol"])
    rows = eng.run(w["n_doublings"])
    compare_rows(rows, gd["rows"])
    for g, o in zip(rows, gd["rows"]):
        assert bonds_close(g["max_bond"], max(o["bond_dims"]))
        # rho^T rho is symmetric; its compression is symmetric up to the
        # truncation: ||rho - rho^T|| <= 2 ||rho - P(rho^T rho)|| gives a
        # defect bound of 2 sqrt(discarded weight) (the oracle itself shows
        # 1e-2 at D* = 12, where the cut falls inside degenerate singular
        # values), and untruncated rows sit at the FP64 resolution of the
        # difference form (~1.5e-8)
        bound = max(1e-6, 2.0 * (o.get("trunc") or 0.0) ** 0.5)
        assert g["herm_defect"] <= bound and o["herm"] <= bound, \
            (o["beta"], g["herm_defect"], o["herm"], bound)


def test_untruncated_L8_matches_exact_diagonalisation(eng_cls):
    from oracle import exact as ex
    from oracle import hamiltonian as oh
    gd = golden("xxz_L8_D256_fp64")
    w = gd["workload"]
    eng = eng_cls.xxz(w["L"], w["J"], w["Delta"], tau0=w["tau0"], dstar=w["dstar"],
                      sweeps=w["sweeps"], order=w["order"])
    rows = eng.run(w["n_doublings"])
    compare_rows(rows, gd["rows"])
    E = ex.ed_spectrum(oh.dense_xxz(w["L"], w["J"], w["Delta"]))
    for g in rows:
        e = ex.ed_thermo(E, g["beta"], w["L"])
        assert abs(g["f"] - e["f"]) <= 1e-10 * abs(e["f"])
        assert abs(g["u"] - e["u"]) <= 1e-10
        assert abs(g["c"] - e["c"]) <= 1e-9


def test_init_state_matches_oracle_densely(eng_cls):
    from oracle import hamiltonian as oh
    from oracle import xtrg as ox
    L, D, tau0 = 6, 0.55, 2.0 ** -7
    eng = eng_cls.xxz(L, 1.0, D, tau0=tau0, dstar=64, sweeps=2, order=4)
    eng.init()
    sites, lnc, beta = eng.get_state()
    rho, lnc_o = ox.init_rho(oh.xxz_chain_mpo(L, 1.0, D), tau0, 4, 64, 2, 1e-15)
    assert beta == tau0
    for a, b in zip(sites, rho):
        assert bonds_close(a.shape[3], b.shape[3])
    A = np.exp(lnc) * oh.mpo_to_dense(sites)
    B = np.exp(lnc_o) * oh.mpo_to_dense(rho)
    assert np.abs(A - B).max() <= 1e-13 * np.abs(B).max()


def test_one_doubling_from_a_given_state(eng_cls):
    """Feed the oracle's rho_n to the GPU and double once on both sides."""
    from oracle import hamiltonian as oh
    from oracle import xtrg as ox
    L, D, tau0 = 7, 1.0, 2.0 ** -5
    H = oh.xxz_chain_mpo(L, 1.0, D)
    rows, states = ox.run_xtrg(H, tau0, 4, 20, 2, 3, 1e-15, keep_states=True)
    rho, lnc = states[-1]
    beta = rows[-1]["beta"]
    eng = eng_cls.xxz(L, 1.0, D, tau0=tau0, dstar=20, sweeps=2, order=4)
    eng.set_state(rho, lnc, beta)
    eng.double()
    g = eng.observables()
    r2, lnc2 = ox.double(rho, lnc, 20, 2, 1e-15)
    o = ox.observables(H, r2, lnc2, 2 * beta, L)
    assert abs(g["lnZ"] - o["lnZ"]) <= 1e-11 * abs(o["lnZ"])
    assert abs(g["u"] - o["u"]) <= 1e-11
    sites, lncg, _ = eng.get_state()
    A = np.exp(lncg) * oh.mpo_to_dense(sites)
    B = np.exp(lnc2) * oh.mpo_to_dense(r2)
    assert np.abs(A - B).max() <= 1e-11 * np.abs(B).max()


@pytest.mark.parametrize("L,dstar,order,sweeps", [(2, 4, 4, 1), (3, 1, 2, 1), (6, 1, 4, 2),
                                                  (5, 64, 1, 3)])
def test_edge_cases(eng_cls, L, dstar, order, sweeps):
    """Shortest chain, D* = 1 (everything truncated to a product operator;
    the leading singular value is non-degenerate), linear initialisation
    (Nc = 1), odd lengths."""
    from oracle import hamiltonian as oh
    from oracle import xtrg as ox
    tau0, nd = 2.0 ** -6, 6
    eng = eng_cls.xxz(L, 1.0, 0.9, tau0=tau0, dstar=dstar, sweeps=sweeps, order=order)
    rows = eng.run(nd)
    ref = ox.run_xtrg(oh.xxz_chain_mpo(L, 1.0, 0.9), tau0, order, dstar, sweeps, nd, 1e-15)
    compare_rows(rows, ref, 1e-9, 1e-9, 1e-8)


def test_errors_are_reported(eng_cls):
    from paper_1801_00142_gb300 import _lib
    eng = eng_cls.xxz(4, 1.0, 1.0, tau0=0.01, dstar=8, sweeps=1)
    with pytest.raises(_lib.XtrgError) as e:
        eng.double()          # before init
    assert e.value.status == _lib.XTRG_EINVAL
    assert "before xtrg_init" in _lib.xtrg_last_error(eng.ctx)
    eng.init()
    big = [np.ones((1, 2, 2, 40)), np.ones((40, 2, 2, 40)), np.ones((40, 2, 2, 1)), np.ones((1, 2, 2, 1))]
    with pytest.raises(_lib.XtrgError):
        eng.set_state(big, 0.0, 1.0)   # bond above the capacity D* + 1


def test_hermiticity_defect_matches_oracle_on_a_nonsymmetric_state(eng_cls):
    """xtrg_observables' herm_defect = ||rho - rho^T||_F / ||rho||_F against the
    oracle's transfer contraction (pinned on dense operators) for a state
    that is not symmetric: rho = I + 0.2 R with R a random MPO, so Tr rho > 0
    and the defect is O(0.1).  A symmetrised state gives ~0."""
    from oracle import hamiltonian as oh
    from oracle import xtrg as ox
    rng = np.random.default_rng(5)
    L = 6
    dims = [1, 3, 4, 5, 4, 3, 1]
    R = [0.5 * rng.standard_normal((dims[i], 2, 2, dims[i + 1])) for i in range(L)]
    W = ox.direct_sum(R, 0.2, oh.identity_mpo(L))
    S = ox.direct_sum(W, 1.0, [w.transpose(0, 2, 1, 3) for w in W])
    H = oh.xxz_chain_mpo(L, 1.0, 1.0)
    eng = eng_cls.xxz(L, 1.0, 1.0, tau0=2.0 ** -8, dstar=16, sweeps=2)
    for state, symmetric in ((W, False), (S, True)):
        ref = ox.observables(H, state, 0.0, 1.0, L)
        eng.set_state(state, 0.0, 1.0)
        g = eng.observables()
        print("herm gpu", g["herm_defect"], "oracle", ref["herm"])
        assert abs(g["lnZ"] - ref["lnZ"]) <= 1e-12 * max(1.0, abs(ref["lnZ"]))
        if symmetric:
            # the square root of a rounding-level difference on both sides
            assert g["herm_defect"] < 1e-7 and ref["herm"] < 1e-7
        else:
            assert ref["herm"] > 0.05
            assert abs(g["herm_defect"] - ref["herm"]) <= 1e-10 + 1e-9 * ref["herm"]
