"""Engine handle: device workspace and stream from PyTorch, work in the C ABI.

PyTorch only allocates the workspace and supplies the CUDA stream; all
arithmetic runs in ``libxtrg.so``.
"""
from __future__ import annotations

import torch

from . import _lib
from .hamiltonians import xxz_bonds_mpo, xxz_chain


class XTRG:
    """One XTRG run: ``init()``, then ``double()`` repeatedly; ``observables()``
    returns the thermodynamics of Eq. ThermalQuan at the current beta."""

    def __init__(self, H_dims, H_sites, tau0, dstar, sweeps=4, order=4, init_sweeps=None,
                 prec="fp64", beta_switch=0.0, svd_rel_tol=1e-15, device="cuda:0", stream=None,
                 keep_parts=True):
        if not torch.cuda.is_available():
            raise RuntimeError("the XTRG engine needs a CUDA device")
        self.L = len(H_sites)
        self.device = torch.device(device)
        self._H = _lib.MpoArgs(H_dims, H_sites)
        self.cfg = _lib.make_config(tau0, order, dstar, sweeps, init_sweeps, prec, beta_switch,
                                    svd_rel_tol, keep_parts)
        nbytes = _lib.xtrg_workspace_bytes(self._H, self.cfg)
        if nbytes == 0:
            raise _lib.XtrgError(_lib.XTRG_EINVAL, "bad Hamiltonian or configuration")
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
            self.stream = stream or torch.cuda.current_stream(self.device)
        ptr = self.workspace.data_ptr()
        ptr = (ptr + 255) // 256 * 256
        self.ctx = _lib.xtrg_create(self._H, self.cfg, ptr, nbytes, self.stream.cuda_stream)

    @classmethod
    def xxz(cls, L, J=1.0, Delta=1.0, **kw):
        dims, sites = xxz_chain(L, J, Delta)
        return cls(dims, sites, **kw)

    @classmethod
    def from_bonds(cls, N, bonds, **kw):
        """H = sum over bonds (i, j, J, Delta) on N sites, e.g. a snake-mapped
        2D lattice (``workloads.square_snake_bonds``)."""
        dims, sites = xxz_bonds_mpo(N, bonds)
        return cls(dims, sites, **kw)

    def init(self):
        _lib.xtrg_init(self.ctx)

    def double(self):
        _lib.xtrg_double(self.ctx)

    def trace(self):
        return _lib.xtrg_trace(self.ctx)

    def observables(self):
        return _lib.xtrg_observables(self.ctx)

    def entanglement(self):
        """MPO entanglement S_E of the current rho at bonds 1..L-1 (Eq. purif)."""
        return _lib.xtrg_entanglement(self.ctx, self.L)

    def get_state(self):
        return _lib.xtrg_get_state(self.ctx, self.L)

    def set_state(self, sites, lnc, beta, right_canonical=False):
        _lib.xtrg_set_state(self.ctx, sites, lnc, beta, right_canonical)

    def checkpoint(self, buf=None):
        """Save the current state into a device buffer (a uint8 tensor on this
        engine's device, allocated here when not given) and return it."""
        import torch
        n = _lib.xtrg_checkpoint_bytes(self.ctx)
        if buf is None:
            buf = torch.empty(n + 256, dtype=torch.uint8, device=self.device)
        ptr = (buf.data_ptr() + 255) // 256 * 256
        if buf.data_ptr() + buf.numel() < ptr + n:
            raise ValueError(f"checkpoint buffer needs {n} bytes after 256-byte alignment")
        _lib.xtrg_checkpoint_save(self.ctx, ptr, n)
        return buf

    def restore(self, buf):
        """Make the state saved in buf (by ``checkpoint``) the current one."""
        ptr = (buf.data_ptr() + 255) // 256 * 256
        _lib.xtrg_checkpoint_load(self.ctx, ptr, buf.data_ptr() + buf.numel() - ptr)

    def counters(self):
        return _lib.xtrg_get_stats(self.ctx)

    def set_profiling(self, on=True):
        _lib.xtrg_set_profiling(self.ctx, on)

    def close(self):
        if getattr(self, "ctx", None):
            _lib.xtrg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, n_doublings):
        """init, then n_doublings doublings; one observables row per beta."""
        self.init()
        rows = [self.observables()]
        for _ in range(n_doublings):
            self.double()
            rows.append(self.observables())
        return rows
