"""CPU check of the product-side operator MPOs for the Binder ratio (Sec. IV
D, Eq. Binder): (S^z_tot)^p with bond p + 1 against the oracle's dense
operator."""
import numpy as np

from oracle import hamiltonian as hm
from paper_1801_00142_gb300.hamiltonians import magnetization_power


def test_magnetization_powers_are_exact_with_bond_p_plus_1():
    for L in (2, 3, 7):
        M = hm.dense_magnetization(L)
        for p in (1, 2, 3, 4):
            dims, sites = magnetization_power(L, p)
            assert max(dims) == p + 1
            want = np.linalg.matrix_power(M, p)
            assert np.abs(hm.mpo_to_dense(sites) - want).max() < 1e-13 * max(1.0, np.abs(want).max())
