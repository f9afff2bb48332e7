"""Interleaved beta grids (z-shifts, Eq. zshift) run concurrently on one GPU.

Each grid tau0_i = tau0 * 2^(i/n_z) is an independent XTRG run with its own
engine, workspace and CUDA stream; one host thread drives each engine (the C
ABI releases the GIL through ctypes), so the grids' kernels overlap on the
device.  The merged rows feed the log-derivative thermodynamics of
``thermo.log_derivative_thermo``.
"""
from __future__ import annotations

import threading

import torch

from .engine import XTRG


def run_zshift(L, J, Delta, tau0, n_z, n_doublings, dstar, sweeps=4, order=4, prec="fp64",
               beta_switch=0.0, device="cuda:0"):
    """Returns a list of n_z row lists (one per grid), each with n_doublings+1
    rows of observables."""
    dev = torch.device(device)
    engines = []
    for i in range(n_z):
        s = torch.cuda.Stream(device=dev)
        engines.append(XTRG.xxz(L, J, Delta, tau0=tau0 * 2.0 ** (i / n_z), dstar=dstar,
                                sweeps=sweeps, order=order, prec=prec, beta_switch=beta_switch,
                                device=device, stream=s))
    out = [None] * n_z
    errs = []

    def work(i):
        try:
            with torch.cuda.device(dev):
                out[i] = engines[i].run(n_doublings)
        except Exception as e:     # re-raised on the calling thread
            errs.append(e)

    threads = [threading.Thread(target=work, args=(i,)) for i in range(n_z)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for e in engines:
        e.close()
    if errs:
        raise errs[0]
    return out
