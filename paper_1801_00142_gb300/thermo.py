"""Thermodynamics on the logarithmic beta grid (host post-processing).

XTRG produces ln Z on beta_n = 2^n tau0; interleaved runs with tau0 shifted by
2^(z_i), z_i = i/n_z (Eq. zshift), fill the grid with spacing
delta ln beta = ln 2 / n_z.  The energy and specific heat then follow from
derivatives with respect to ln beta (Eq. ThermalQuan:X):

    u   = (1/beta) d(beta f)/d ln beta,      beta f = -ln Z / N
    c_V = -beta du/d ln beta

which divide numerical differences by T (not T^2 as du/dT would).  The
derivatives here are second-order three-point differences on the merged grid
(non-uniform in general).
"""
from __future__ import annotations

import numpy as np


def merge_grids(runs):
    """runs: list of lists of rows with 'beta' and 'lnZ'; returns sorted
    arrays (beta, lnZ) of the merged grid."""
    pts = sorted((r["beta"], r["lnZ"]) for rows in runs for r in rows)
    return np.array([p[0] for p in pts]), np.array([p[1] for p in pts])


def _deriv(x, y):
    """dy/dx at every node from the three-point Lagrange interpolant
    (one-sided at the ends)."""
    n = len(x)
    d = np.empty(n)
    for i in range(n):
        j = [0, 1, 2] if i == 0 else ([n - 3, n - 2, n - 1] if i == n - 1 else [i - 1, i, i + 1])
        x0, x1, x2 = x[j]
        y0, y1, y2 = y[j]
        xi = x[i]
        d[i] = (y0 * (2 * xi - x1 - x2) / ((x0 - x1) * (x0 - x2))
                + y1 * (2 * xi - x0 - x2) / ((x1 - x0) * (x1 - x2))
                + y2 * (2 * xi - x0 - x1) / ((x2 - x0) * (x2 - x1)))
    return d


def log_derivative_thermo(beta, lnZ, N):
    """u and c_V per site from ln Z on a logarithmic grid (Eq. ThermalQuan:X)."""
    beta = np.asarray(beta, float)
    lnZ = np.asarray(lnZ, float)
    x = np.log(beta)
    u = _deriv(x, -lnZ / N) / beta
    c = -beta * _deriv(x, u)
    return u, c
