"""Exact thermodynamics for the oracle (test infrastructure only).

* ``ed_thermo``            exact diagonalisation, the paper's reference data
                           for small clusters (Sec. III, Fig. FeErr, Fig. FeSq)
* ``free_fermion_thermo``  closed form of the open XY chain, App. F:
                           eps_k = J cos(k pi / (L+1)), Z = prod_k (1 + e^{-beta eps_k})
* ``two_site_lnZ``         closed form of a single XXZ bond

Thermodynamic quantities follow Eq. ThermalQuan (Sec. III A):
f = -ln Z / (N beta), u = <H>/N, c_V = beta^2 (<H^2> - <H>^2) / N
(the last is -beta^2 du/dbeta written out for a Gibbs state).
"""
from __future__ import annotations

import numpy as np


def ed_spectrum(H: np.ndarray) -> np.ndarray:
    return np.linalg.eigvalsh(H)


def ed_thermo(E: np.ndarray, beta: float, N: int) -> dict:
    """Thermodynamics at inverse temperature beta from the full spectrum E."""
    E = np.asarray(E, dtype=np.float64)
    E0 = E.min()
    w = np.exp(-beta * (E - E0))
    z = w.sum()
    lnZ = -beta * E0 + np.log(z)
    p = w / z
    e1 = float(p @ E)
    dE = E - e1
    var = float(p @ (dE * dE))
    return {"beta": beta, "lnZ": float(lnZ), "f": float(-lnZ / (N * beta)),
            "u": e1 / N, "c": beta * beta * var / N,
            # Z(2 beta) = Tr rho(beta)^2, the Frobenius-norm identity of Sec. II B
            "lnZ2": float(-2 * beta * E0 + np.log(np.sum(w * w)))}


def free_fermion_eps(L: int, J: float = 1.0) -> np.ndarray:
    """One-particle energies of the open tight-binding chain (App. F)."""
    k = np.arange(1, L + 1)
    return J * np.cos(k * np.pi / (L + 1))


def free_fermion_thermo(L: int, beta: float, J: float = 1.0) -> dict:
    """Closed form of App. F for the XY chain (Delta = 0), any L."""
    eps = free_fermion_eps(L, J)
    x = beta * eps
    lnZ = float(np.sum(np.logaddexp(0.0, -x)))            # ln(1 + e^{-x})
    n = 0.5 * (1.0 - np.tanh(0.5 * x))                    # 1 / (1 + e^{x})
    u = float(np.sum(eps * n)) / L
    c = float(beta * beta * np.sum(eps * eps * n * (1.0 - n))) / L
    lnZ2 = float(np.sum(np.logaddexp(0.0, -2.0 * x)))
    return {"beta": beta, "lnZ": lnZ, "f": -lnZ / (L * beta), "u": u, "c": c,
            "lnZ2": lnZ2}


def two_site_lnZ(beta: float, J: float = 1.0, Delta: float = 1.0) -> float:
    """One XXZ bond: triplet-like |uu>,|dd> at J Delta/4, the symmetric and
    antisymmetric combinations of |ud>,|du> at -J Delta/4 +- J/2."""
    E = np.array([J * Delta / 4, J * Delta / 4, -J * Delta / 4 + J / 2, -J * Delta / 4 - J / 2])
    return float(np.log(np.sum(np.exp(-beta * E))))


def high_t_lnZ(L: int, beta: float, J: float = 1.0, Delta: float = 1.0, bonds=None) -> float:
    """ln Z to second order in beta: N ln 2 + beta^2 Tr(H^2) / (2 * 2^N), with
    Tr H = 0 and Tr(H^2)/2^N = sum_bonds J^2 (2 + Delta^2) / 16."""
    nb = (L - 1) if bonds is None else len(bonds)
    return L * np.log(2.0) + 0.5 * beta * beta * nb * J * J * (2.0 + Delta * Delta) / 16.0


def ed_binder(H: np.ndarray, M: np.ndarray, beta: float) -> float:
    """U_4 = <M^2>^2 / <M^4> at inverse temperature beta by exact
    diagonalisation of the dense H (M: dense S^z_tot)."""
    E, V = np.linalg.eigh(H)
    w = np.exp(-beta * (E - E.min()))
    M2 = M @ M
    m2 = float(np.sum(w * np.einsum("ij,ik,kj->j", V, M2, V))) / w.sum()
    m4 = float(np.sum(w * np.einsum("ij,ik,kj->j", V, M2 @ M2, V))) / w.sum()
    return m2 * m2 / m4
