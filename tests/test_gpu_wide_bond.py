"""Bonds wider than one orthonormalisation block on the tensor-core path.

The truncation of the tensor-core path (App. D.1, the two-site split of the
variational compression) orthonormalises the subspace basis block by block:
each column block is projected twice against the blocks before it and then
orthonormalised by scaled CholeskyQR2.  At the default width of 256 columns
that path runs from D* = 257 on; the config's orth_block lets it run on
small bonds too.  Both are checked against the FP64 oracle and against exact
diagonalisation, with the fraction of updates that fell back to the exact
FP64 split bounded (a broken blocked orthonormalisation would hide behind
that fallback)."""
import json
import os

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


@pytest.mark.parametrize("orth_block", [32, 96])
def test_blocked_orthonormalisation_matches_oracle(eng_cls, orth_block):
    """L = 8 Heisenberg, D* = 256 (middle bonds up to 256 columns, i.e. 8
    blocks of 32 or 3 blocks of 96 with a ragged last one) against the
    oracle's FP64 rows, at the bars of the one-block path."""
    with open(os.path.join(HERE, "golden", "oracle_xxz_L8_D256_fp64.json")) as f:
        gd = json.load(f)
    w = gd["workload"]
    eng = eng_cls.xxz(w["L"], w["J"], w["Delta"], tau0=w["tau0"], dstar=w["dstar"],
                      sweeps=w["sweeps"], order=w["order"], prec="bf16x6", beta_switch=2.0,
                      orth_block=orth_block)
    rows = eng.run(w["n_doublings"])
    st = eng.counters()
    worst_f = max(abs(g["f"] - o["f"]) for g, o in zip(rows, gd["rows"]))
    worst_u = max(abs(g["u"] - o["u"]) for g, o in zip(rows, gd["rows"]))
    print("orth_block", orth_block, "max |df|", worst_f, "max |du|", worst_u, "max bond",
          max(r["max_bond"] for r in rows), "fallbacks", st["exact_split_fallbacks"], "of",
          st["two_site_updates"])
    assert max(r["max_bond"] for r in rows) > orth_block
    assert worst_f <= 1e-6
    assert worst_u <= 1e-5
    assert st["exact_split_fallbacks"] <= 0.1 * st["two_site_updates"]


def test_d320_against_exact_diagonalisation(eng_cls):
    """L = 10 Heisenberg at D* = 320: the middle bonds hold 320 columns, two
    blocks (256 + 64), on the tensor cores from beta = 1/4 on; every row
    against exact diagonalisation."""
    import numpy as np
    from oracle import exact as ex
    from oracle import hamiltonian as oh
    L = 10
    E = ex.ed_spectrum(oh.dense_xxz(L, 1.0, 1.0))
    eng = eng_cls.xxz(L, 1.0, 1.0, tau0=2.0 ** -8, dstar=320, sweeps=4, order=4, prec="bf16x6",
                      beta_switch=0.25)
    rows = eng.run(11)
    st = eng.counters()
    mb = max(r["max_bond"] for r in rows)
    print("max bond", mb, "fallbacks", st["exact_split_fallbacks"], "of", st["two_site_updates"])
    assert mb > 256
    assert st["exact_split_fallbacks"] <= 0.1 * st["two_site_updates"]
    for r in rows:
        ref = ex.ed_thermo(E, r["beta"], L)
        print(f"beta={r['beta']:9.5f} |df| {abs(r['f'] - ref['f']):.2e} |du| "
              f"{abs(r['u'] - ref['u']):.2e} trunc {r['trunc_err']:.1e}")
        assert abs(r["f"] - ref["f"]) <= 1e-6 + r["trunc_err"], (r["beta"], r["f"], ref["f"])
        assert abs(r["u"] - ref["u"]) <= 1e-5 + r["trunc_err"], (r["beta"], r["u"], ref["u"])
    assert np.isfinite(rows[-1]["c"])
