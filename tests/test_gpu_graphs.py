"""Graph-captured tensor-core doublings.

Once the bonds are saturated, xtrg_double captures the device work of a
doubling (Sec. II B, Eq. rho:scale2; the sweeps of App. D.1 with every
decision, the exact-split fallback included, taken on the device) as a CUDA
graph per buffer parity and replays it.  A replay must compute exactly what a
direct run computes: the rows of a run with graphs and of one without are
compared bit for bit, and both against the free-fermion closed form (App. F).
"""
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


def _run(eng_cls, graphs, L=16, dstar=64, n=14):
    eng = eng_cls.xxz(L, 1.0, 0.0, tau0=2.0 ** -8, dstar=dstar, sweeps=2, order=4, prec="bf16x6",
                      beta_switch=0.25)
    eng.set_graphs(graphs)
    rows = eng.run(n)
    st = eng.counters()
    eng.close()
    return rows, st


def test_graph_replay_is_bit_identical_to_direct_run(eng_cls):
    from oracle import exact as ex
    g_rows, g_st = _run(eng_cls, True)
    d_rows, d_st = _run(eng_cls, False)
    print("captures", g_st["graph_captures"], "replays", g_st["graph_replays"])
    assert g_st["graph_captures"] >= 1 and g_st["graph_replays"] >= 2
    assert d_st["graph_captures"] == 0 and d_st["graph_replays"] == 0
    for g, d in zip(g_rows, d_rows):
        for key in ("beta", "lnZ", "f", "u", "c", "max_bond"):
            assert g[key] == d[key], (key, g["beta"], g[key], d[key])
        # the discarded weight 1 - ||kept||^2 / ||C_E||^2 comes from sums with
        # atomic (order-dependent) accumulation, and the subtraction magnifies
        # their last-bit differences
        assert abs(g["trunc_err"] - d["trunc_err"]) <= 1e-14, (g["beta"], g["trunc_err"])
    for key in ("two_site_updates", "exact_split_fallbacks", "contraction_flops"):
        assert g_st[key] == d_st[key], key
    # sanity against the closed form (D* = 64 truncates this chain: the
    # accuracy gate itself is tested at D* = 256 elsewhere)
    for r in g_rows:
        e = ex.free_fermion_thermo(16, r["beta"])
        assert abs(r["f"] - e["f"]) <= 1e-5, (r["beta"], r["f"], e["f"])


def test_graphs_follow_a_new_state(eng_cls):
    """set_state between doublings: a replayed graph reads the buffers it was
    captured on at replay time, so a new right-canonical state with the same
    bonds (the saturated state of another chain) is doubled exactly as a
    direct run doubles it."""
    kw = dict(tau0=2.0 ** -8, dstar=48, sweeps=2, order=4, prec="bf16x6", beta_switch=0.25)
    eng = eng_cls.xxz(12, 1.0, 0.0, **kw)
    eng.run(14)
    assert eng.counters()["graph_captures"] >= 2
    other = eng_cls.xxz(12, 1.0, 0.5, **kw)
    other.set_graphs(False)
    other.run(14)
    sites, lnc, beta = other.get_state()
    ref = eng_cls.xxz(12, 1.0, 0.0, **kw)
    ref.set_graphs(False)
    ref.run(14)
    r0 = eng.counters()["graph_replays"]
    for e in (eng, ref):
        e.set_state(sites, lnc, beta, right_canonical=True)
        e.double()
    assert eng.counters()["graph_replays"] == r0 + 1
    a, b = eng.observables(), ref.observables()
    assert a["lnZ"] == b["lnZ"] and a["u"] == b["u"]
    assert abs(a["trunc_err"] - b["trunc_err"]) <= 1e-14


def test_hermiticity_diagnostic_can_be_switched_off(eng_cls):
    """Without the FP64 Hermiticity transfers, observables() reports NaN for
    herm_defect and the same thermodynamics (the traces are separate)."""
    import math
    eng = eng_cls.xxz(10, 1.0, 1.0, tau0=2.0 ** -6, dstar=64, sweeps=2, order=4)
    eng.run(4)
    on = eng.observables()
    eng.set_herm_check(False)
    off = eng.observables()
    assert math.isnan(off["herm_defect"]) and math.isfinite(on["herm_defect"])
    for key in ("lnZ", "f", "u", "c", "lnZ2", "max_bond"):
        assert on[key] == off[key], key
