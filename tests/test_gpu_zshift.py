"""Concurrent z-shift grids (Eq. zshift): each grid's ln Z equals the oracle's
for its own tau0, and the log-derivative u, c_V on the merged grid agree with
exact diagonalisation to the finite-difference accuracy of the grid."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_zshift_grids_match_oracle_and_ed():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_00142_gb300.build import build
    build()
    from paper_1801_00142_gb300.zshift import run_zshift
    from paper_1801_00142_gb300.thermo import merge_grids, log_derivative_thermo
    from oracle import exact as ex
    from oracle import hamiltonian as oh
    from oracle import xtrg as ox

    L, Delta, nz, tau0, nd = 6, 1.0, 4, 2.0 ** -8, 10
    runs = run_zshift(L, 1.0, Delta, tau0, nz, nd, dstar=64, sweeps=2)
    for i, rows in enumerate(runs):
        H = oh.xxz_chain_mpo(L, 1.0, Delta)
        ref = ox.run_xtrg(H, tau0 * 2.0 ** (i / nz), 4, 64, 2, nd, 1e-15)
        for g, o in zip(rows, ref):
            assert abs(g["lnZ"] - o["lnZ"]) <= 1e-10 * max(1.0, abs(o["lnZ"]))
    beta, lnZ = merge_grids(runs)
    u, c = log_derivative_thermo(beta, lnZ, L)
    E = ex.ed_spectrum(oh.dense_xxz(L, 1.0, Delta))
    ref_u = np.array([ex.ed_thermo(E, b, L)["u"] for b in beta])
    ref_c = np.array([ex.ed_thermo(E, b, L)["c"] for b in beta])
    inner = slice(2, -2)
    assert np.abs(u[inner] - ref_u[inner]).max() < 1e-2
    assert np.abs(c[inner] - ref_c[inner]).max() < 2e-2
