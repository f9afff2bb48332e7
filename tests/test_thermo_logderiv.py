"""The log-derivative estimator of Eq. ThermalQuan:X against the free-fermion
closed form (App. F): u and c_V recovered from ln Z on interleaved z-shift
grids, to the finite-difference accuracy of the grid."""
import numpy as np

from oracle import exact as ex
from paper_1801_00142_gb300.thermo import log_derivative_thermo, merge_grids


def test_interleaved_grids_recover_u_and_c():
    L, nz = 32, 16
    runs = []
    for i in range(nz):
        tau0 = 2.0 ** -6 * 2.0 ** (i / nz)
        runs.append([{"beta": tau0 * 2 ** n, "lnZ": ex.free_fermion_thermo(L, tau0 * 2 ** n)["lnZ"]}
                     for n in range(11)])
    beta, lnZ = merge_grids(runs)
    assert np.all(np.diff(np.log(beta)) > 0)
    u, c = log_derivative_thermo(beta, lnZ, L)
    inner = slice(2, -2)
    ref_u = np.array([ex.free_fermion_thermo(L, b)["u"] for b in beta])
    ref_c = np.array([ex.free_fermion_thermo(L, b)["c"] for b in beta])
    assert np.abs(u[inner] - ref_u[inner]).max() < 2e-3
    assert np.abs(c[inner] - ref_c[inner]).max() < 5e-3


def test_grid_refinement_converges_at_second_order():
    L = 16
    errs = []
    for nz in (8, 16, 32):
        beta = np.array([2.0 ** (k / nz) for k in range(-nz * 2, nz * 3)])
        lnZ = np.array([ex.free_fermion_thermo(L, b)["lnZ"] for b in beta])
        u, _ = log_derivative_thermo(beta, lnZ, L)
        ref = np.array([ex.free_fermion_thermo(L, b)["u"] for b in beta])
        errs.append(np.abs(u - ref)[3:-3].max())
    assert errs[1] < errs[0] / 3 and errs[2] < errs[1] / 3
