"""xtrg_batch_run on one GPU: instances of uneven size (chain length, Delta,
D*, tau0 grid) run concurrently from one workspace; every instance's rows
equal the oracle's for that instance (FP64 path, 1e-10)."""
import pytest

pytestmark = pytest.mark.gpu


def test_batch_matches_oracle_per_instance():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_00142_gb300.build import build
    build()
    from oracle import hamiltonian as oh
    from oracle import xtrg as ox
    from paper_1801_00142_gb300.batch import run_batch
    from paper_1801_00142_gb300.hamiltonians import xxz_chain

    cases = [(6, 1.0, 2.0 ** -8, 64, 8), (5, 0.4, 2.0 ** -8 * 2 ** 0.5, 32, 7),
             (8, 0.0, 2.0 ** -7, 64, 6), (4, 1.3, 2.0 ** -6, 16, 9)]
    items = []
    for L, D, tau0, dstar, nd in cases:
        dims, sites = xxz_chain(L, 1.0, D)
        items.append((dims, sites, nd, dict(tau0=tau0, order=4, dstar=dstar, sweeps=2)))
    rows = run_batch(items, max_concurrent=3)
    assert [len(r) for r in rows] == [nd + 1 for *_, nd in cases]
    for (L, D, tau0, dstar, nd), got in zip(cases, rows):
        ref = ox.run_xtrg(oh.xxz_chain_mpo(L, 1.0, D), tau0, 4, dstar, 2, nd, 1e-15)
        for g, o in zip(got, ref):
            assert abs(g["beta"] - o["beta"]) < 1e-14 * o["beta"]
            assert abs(g["lnZ"] - o["lnZ"]) <= 1e-10 * max(1.0, abs(o["lnZ"]))
            assert abs(g["u"] - o["u"]) <= 1e-10


def test_batch_tensor_core_path_matches_oracle_per_instance():
    """The batched runner with split-BF16 contractions (bf16x6; doublings
    from beta >= 1/4 on the tensor cores): uneven instances run three at a
    time, each within the mixed-precision gate of the FP64 oracle,
    |df|/site <= 1e-6 and |du| <= 1e-5 at every beta (untruncated D*, so
    the oracle's rows are the exact thermodynamics of the instance)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_00142_gb300.build import build
    build()
    from oracle import hamiltonian as oh
    from oracle import xtrg as ox
    from paper_1801_00142_gb300.batch import run_batch
    from paper_1801_00142_gb300.hamiltonians import xxz_chain

    cases = [(6, 1.0, 2.0 ** -8, 64, 10), (7, 0.4, 2.0 ** -8 * 2 ** 0.5, 64, 9),
             (8, 0.0, 2.0 ** -7, 256, 9), (5, 1.3, 2.0 ** -6, 16, 8)]
    items = []
    for L, D, tau0, dstar, nd in cases:
        dims, sites = xxz_chain(L, 1.0, D)
        items.append((dims, sites, nd, dict(tau0=tau0, order=4, dstar=dstar, sweeps=2,
                                            prec="bf16x6", beta_switch=0.25)))
    rows = run_batch(items, max_concurrent=3)
    for (L, D, tau0, dstar, nd), got in zip(cases, rows):
        ref = ox.run_xtrg(oh.xxz_chain_mpo(L, 1.0, D), tau0, 4, dstar, 2, nd, 1e-15)
        assert len(got) == nd + 1
        for g, o in zip(got, ref):
            assert abs(g["f"] - o["f"]) <= 1e-6, (L, o["beta"], g["f"], o["f"])
            assert abs(g["u"] - o["u"]) <= 1e-5, (L, o["beta"], g["u"], o["u"])
