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
                 keep_parts=True, orth_block=0):
        if not torch.cuda.is_available():
            raise RuntimeError("the XTRG engine needs a CUDA device")
        self.L = len(H_sites)
        self.device = torch.device(device)
        self._H = _lib.MpoArgs(H_dims, H_sites)
        self.cfg = _lib.make_config(tau0, order, dstar, sweeps, init_sweeps, prec, beta_switch,
                                    svd_rel_tol, keep_parts, orth_block)
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

    def settn_step(self, dtau, order):
        """rho(beta) -> rho(beta + dtau) by the pointwise-Taylor series of
        Eq. Tay to the given order (FP64; see xtrg_settn_step)."""
        import torch
        n = _lib.xtrg_settn_workspace_bytes(self.ctx, order)
        buf = torch.empty(n + 256, dtype=torch.uint8, device=self.device)
        ptr = (buf.data_ptr() + 255) // 256 * 256
        _lib.xtrg_settn_step(self.ctx, dtau, order, ptr, n)
        del buf

    def run_settn(self, n_steps, order):
        """init, then n_steps pointwise-Taylor steps along tau_n = 2^n tau0
        (dtau = tau_n); one observables row per grid point."""
        self.init()
        rows = [self.observables()]
        for _ in range(n_steps):
            self.settn_step(rows[-1]["beta"], order)
            rows.append(self.observables())
        return rows

    def expectation(self, dims, sites):
        """<O> = Tr(O rho)/Tr rho for an operator MPO (bond dims, sites)."""
        return _lib.xtrg_expectation(self.ctx, _lib.MpoArgs(dims, sites))

    def binder_ratio(self):
        """U_4 = <M^2>^2 / <M^4> with M = S^z_tot (Sec. IV D, Eq. Binder)."""
        from .hamiltonians import magnetization_power
        m2 = self.expectation(*magnetization_power(self.L, 2))
        return m2 * m2 / self.expectation(*magnetization_power(self.L, 4))

    def cross_product(self, ckpt_a, ckpt_b):
        """Make rho_a rho_b (two buffers from ``checkpoint``) the current
        state: rho at beta_a + beta_b (Sec. II B, after Eq. zshift)."""
        pa = (ckpt_a.data_ptr() + 255) // 256 * 256
        pb = (ckpt_b.data_ptr() + 255) // 256 * 256
        _lib.xtrg_cross_product(self.ctx, pa, ckpt_a.data_ptr() + ckpt_a.numel() - pa,
                                pb, ckpt_b.data_ptr() + ckpt_b.numel() - pb)

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

    def set_herm_check(self, on=True):
        """Compute (default) or skip the Hermiticity diagnostic in
        observables() (herm_defect is NaN when skipped)."""
        _lib.xtrg_set_herm_check(self.ctx, on)

    def set_graphs(self, on=True):
        """Allow (default) or forbid replaying saturated tensor-core doublings
        from captured CUDA graphs."""
        _lib.xtrg_set_graphs(self.ctx, on)

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
