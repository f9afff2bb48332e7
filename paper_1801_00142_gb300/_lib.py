"""ctypes binding of the C ABI declared in include/xtrg.h.

Argument marshalling only: every step of the XTRG path runs in the CUDA
library.  Importing this module loads ``libxtrg.so`` and fails loudly if it
has not been built (there is no fallback implementation).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libxtrg.so")

XTRG_OK, XTRG_EINVAL, XTRG_ENOMEM, XTRG_ECUDA, XTRG_ENUMERIC, XTRG_ETIMEOUT = range(6)
XTRG_FP64, XTRG_BF16X6, XTRG_BF16X3 = 0, 1, 2
PRECISIONS = {"fp64": XTRG_FP64, "bf16x6": XTRG_BF16X6, "bf16x3": XTRG_BF16X3}
STATUS_NAMES = {0: "XTRG_OK", 1: "XTRG_EINVAL", 2: "XTRG_ENOMEM", 3: "XTRG_ECUDA",
                4: "XTRG_ENUMERIC", 5: "XTRG_ETIMEOUT"}

# every exported symbol the header declares
SYMBOLS = ["xtrg_workspace_bytes", "xtrg_create", "xtrg_init", "xtrg_double", "xtrg_trace",
           "xtrg_observables", "xtrg_get_state", "xtrg_set_state", "xtrg_get_stats",
           "xtrg_set_profiling", "xtrg_set_graphs", "xtrg_set_herm_check",
           "xtrg_last_error", "xtrg_destroy", "xtrg_tc_gemm_workspace_bytes", "xtrg_tc_gemm",
           "xtrg_tc_gemm_static", "xtrg_batch_plan", "xtrg_batch_run", "xtrg_checkpoint_bytes",
           "xtrg_checkpoint_save", "xtrg_checkpoint_load", "xtrg_entanglement",
           "xtrg_tc_gemm_nn_workspace_bytes", "xtrg_tc_gemm_nn", "xtrg_settn_workspace_bytes",
           "xtrg_settn_step", "xtrg_expectation", "xtrg_cross_product"]


class xtrg_mpo(C.Structure):
    _fields_ = [("L", C.c_int), ("d", C.c_int), ("bond_dims", C.POINTER(C.c_int)),
                ("W", C.POINTER(C.POINTER(C.c_double)))]


class xtrg_config(C.Structure):
    _fields_ = [("tau0", C.c_double), ("order", C.c_int), ("dstar", C.c_int),
                ("sweeps", C.c_int), ("init_sweeps", C.c_int), ("prec", C.c_int),
                ("beta_switch", C.c_double), ("svd_rel_tol", C.c_double),
                ("keep_parts", C.c_int), ("orth_block", C.c_int)]


class xtrg_obs(C.Structure):
    _fields_ = [("beta", C.c_double), ("lnZ", C.c_double), ("f", C.c_double),
                ("u", C.c_double), ("c", C.c_double), ("lnZ2", C.c_double),
                ("trunc_err", C.c_double), ("herm_defect", C.c_double),
                ("max_bond", C.c_int), ("n_doublings", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class xtrg_stats(C.Structure):
    _fields_ = [("contraction_flops", C.c_double), ("split_flops", C.c_double),
                ("tc_flops", C.c_double), ("tc_ms", C.c_double),
                ("two_site_updates", C.c_longlong), ("tc_launches", C.c_longlong),
                ("kernel_launches", C.c_longlong), ("exact_split_fallbacks", C.c_longlong),
                ("split_ms", C.c_double), ("orth_cluster_calls", C.c_longlong),
                ("fp64_update_ms", C.c_double), ("fp64_updates_timed", C.c_longlong),
                ("fp64_env_pass_ms", C.c_double), ("orth_fallbacks", C.c_longlong),
                ("orth_full_second_pass", C.c_longlong), ("orth_deflated_columns", C.c_longlong),
                ("graph_captures", C.c_longlong),
                ("graph_replays", C.c_longlong), ("split_shapes_tuned", C.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class XtrgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(LIB_PATH)
    P = C.c_void_p
    lib.xtrg_workspace_bytes.restype = C.c_size_t
    lib.xtrg_workspace_bytes.argtypes = [C.POINTER(xtrg_mpo), C.POINTER(xtrg_config)]
    lib.xtrg_create.restype = C.c_int
    lib.xtrg_create.argtypes = [C.POINTER(P), C.POINTER(xtrg_mpo), C.POINTER(xtrg_config), P,
                                C.c_size_t, P]
    for name in ("xtrg_init", "xtrg_double"):
        getattr(lib, name).restype = C.c_int
        getattr(lib, name).argtypes = [P]
    lib.xtrg_trace.restype = C.c_int
    lib.xtrg_trace.argtypes = [P, C.POINTER(C.c_double)]
    lib.xtrg_observables.restype = C.c_int
    lib.xtrg_observables.argtypes = [P, C.POINTER(xtrg_obs)]
    lib.xtrg_get_state.restype = C.c_int
    lib.xtrg_get_state.argtypes = [P, C.POINTER(C.c_int), C.POINTER(C.POINTER(C.c_double)),
                                   C.POINTER(C.c_double), C.POINTER(C.c_double)]
    lib.xtrg_set_state.restype = C.c_int
    lib.xtrg_set_state.argtypes = [P, C.POINTER(xtrg_mpo), C.c_double, C.c_double, C.c_int]
    lib.xtrg_get_stats.restype = C.c_int
    lib.xtrg_get_stats.argtypes = [P, C.POINTER(xtrg_stats)]
    lib.xtrg_set_profiling.restype = C.c_int
    lib.xtrg_set_profiling.argtypes = [P, C.c_int]
    lib.xtrg_set_graphs.restype = C.c_int
    lib.xtrg_set_graphs.argtypes = [P, C.c_int]
    lib.xtrg_set_herm_check.restype = C.c_int
    lib.xtrg_set_herm_check.argtypes = [P, C.c_int]
    lib.xtrg_batch_plan.restype = C.c_int
    lib.xtrg_batch_plan.argtypes = [C.c_int, C.POINTER(xtrg_mpo), C.POINTER(xtrg_config),
                                    C.c_size_t, C.c_int, C.POINTER(C.c_int),
                                    C.POINTER(C.c_size_t)]
    lib.xtrg_batch_run.restype = C.c_int
    lib.xtrg_batch_run.argtypes = [C.c_int, C.POINTER(xtrg_mpo), C.POINTER(xtrg_config),
                                   C.POINTER(C.c_int), C.POINTER(xtrg_obs), P, C.c_size_t,
                                   C.c_int, P]
    lib.xtrg_last_error.restype = C.c_char_p
    lib.xtrg_last_error.argtypes = [P]
    lib.xtrg_destroy.restype = None
    lib.xtrg_destroy.argtypes = [P]
    lib.xtrg_tc_gemm_workspace_bytes.restype = C.c_size_t
    lib.xtrg_tc_gemm_workspace_bytes.argtypes = [C.c_int] * 6
    lib.xtrg_tc_gemm.restype = C.c_int
    lib.xtrg_tc_gemm.argtypes = [P, P, P] + [C.c_int] * 7 + [P, C.c_size_t, P]
    lib.xtrg_expectation.restype = C.c_int
    lib.xtrg_expectation.argtypes = [P, C.POINTER(xtrg_mpo), C.POINTER(C.c_double)]
    lib.xtrg_cross_product.restype = C.c_int
    lib.xtrg_cross_product.argtypes = [P, P, C.c_size_t, P, C.c_size_t]
    lib.xtrg_settn_workspace_bytes.restype = C.c_size_t
    lib.xtrg_settn_workspace_bytes.argtypes = [P, C.c_int]
    lib.xtrg_settn_step.restype = C.c_int
    lib.xtrg_settn_step.argtypes = [P, C.c_double, C.c_int, P, C.c_size_t]
    lib.xtrg_entanglement.restype = C.c_int
    lib.xtrg_entanglement.argtypes = [P, C.POINTER(C.c_double), C.c_int]
    lib.xtrg_checkpoint_bytes.restype = C.c_size_t
    lib.xtrg_checkpoint_bytes.argtypes = [P]
    lib.xtrg_checkpoint_save.restype = C.c_int
    lib.xtrg_checkpoint_save.argtypes = [P, P, C.c_size_t]
    lib.xtrg_checkpoint_load.restype = C.c_int
    lib.xtrg_checkpoint_load.argtypes = [P, P, C.c_size_t]
    lib.xtrg_tc_gemm_nn_workspace_bytes.restype = C.c_size_t
    lib.xtrg_tc_gemm_nn_workspace_bytes.argtypes = [C.c_int] * 6
    lib.xtrg_tc_gemm_nn.restype = C.c_int
    lib.xtrg_tc_gemm_nn.argtypes = [P, P, P] + [C.c_int] * 7 + [P, C.c_size_t, P]
    lib.xtrg_tc_gemm_static.restype = C.c_int
    lib.xtrg_tc_gemm_static.argtypes = [P, P, P] + [C.c_int] * 7 + [P]
    return lib


LIB = _load()


class MpoArgs:
    """Keeps the ctypes views of a host MPO alive while a call uses them."""

    def __init__(self, dims, sites):
        self.dims = np.ascontiguousarray(dims, dtype=np.int32)
        self.sites = [np.ascontiguousarray(w, dtype=np.float64) for w in sites]
        L = len(self.sites)
        self.ptrs = (C.POINTER(C.c_double) * L)(
            *[w.ctypes.data_as(C.POINTER(C.c_double)) for w in self.sites])
        self.struct = xtrg_mpo(L, 2, self.dims.ctypes.data_as(C.POINTER(C.c_int)), self.ptrs)


def make_config(tau0, order, dstar, sweeps, init_sweeps=None, prec="fp64", beta_switch=0.0,
                svd_rel_tol=1e-15, keep_parts=True, orth_block=0):
    p = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    return xtrg_config(float(tau0), int(order), int(dstar), int(sweeps),
                       int(init_sweeps or sweeps), p, float(beta_switch), float(svd_rel_tol),
                       int(bool(keep_parts)), int(orth_block))


def _check(ctx, status):
    if status != XTRG_OK:
        msg = LIB.xtrg_last_error(ctx).decode() if ctx else ""
        raise XtrgError(status, msg)


def xtrg_workspace_bytes(H: MpoArgs, cfg: xtrg_config) -> int:
    return int(LIB.xtrg_workspace_bytes(C.byref(H.struct), C.byref(cfg)))


def xtrg_create(H: MpoArgs, cfg: xtrg_config, dev_ptr: int, nbytes: int, stream: int):
    ctx = C.c_void_p()
    s = LIB.xtrg_create(C.byref(ctx), C.byref(H.struct), C.byref(cfg), C.c_void_p(dev_ptr),
                        C.c_size_t(nbytes), C.c_void_p(stream))
    if s != XTRG_OK:
        raise XtrgError(s, "xtrg_create")
    return ctx


def xtrg_init(ctx):
    _check(ctx, LIB.xtrg_init(ctx))


def xtrg_double(ctx):
    _check(ctx, LIB.xtrg_double(ctx))


def xtrg_trace(ctx) -> float:
    v = C.c_double()
    _check(ctx, LIB.xtrg_trace(ctx, C.byref(v)))
    return v.value


def xtrg_observables(ctx) -> dict:
    o = xtrg_obs()
    _check(ctx, LIB.xtrg_observables(ctx, C.byref(o)))
    return o.as_dict()


def xtrg_get_state(ctx, L):
    dims = np.zeros(L + 1, dtype=np.int32)
    lnc, beta = C.c_double(), C.c_double()
    _check(ctx, LIB.xtrg_get_state(ctx, dims.ctypes.data_as(C.POINTER(C.c_int)), None,
                                   C.byref(lnc), C.byref(beta)))
    sites = [np.empty((dims[i], 2, 2, dims[i + 1])) for i in range(L)]
    ptrs = (C.POINTER(C.c_double) * L)(*[w.ctypes.data_as(C.POINTER(C.c_double)) for w in sites])
    _check(ctx, LIB.xtrg_get_state(ctx, dims.ctypes.data_as(C.POINTER(C.c_int)), ptrs,
                                   C.byref(lnc), C.byref(beta)))
    return sites, lnc.value, beta.value


def xtrg_set_state(ctx, sites, lnc, beta, right_canonical=False):
    dims = [1] + [w.shape[3] for w in sites]
    m = MpoArgs(dims, sites)
    _check(ctx, LIB.xtrg_set_state(ctx, C.byref(m.struct), float(lnc), float(beta),
                                   1 if right_canonical else 0))


def xtrg_expectation(ctx, O: MpoArgs) -> float:
    v = C.c_double()
    _check(ctx, LIB.xtrg_expectation(ctx, C.byref(O.struct), C.byref(v)))
    return v.value


def xtrg_cross_product(ctx, ptr_a, bytes_a, ptr_b, bytes_b):
    _check(ctx, LIB.xtrg_cross_product(ctx, C.c_void_p(ptr_a), C.c_size_t(bytes_a),
                                       C.c_void_p(ptr_b), C.c_size_t(bytes_b)))


def xtrg_settn_workspace_bytes(ctx, order) -> int:
    return int(LIB.xtrg_settn_workspace_bytes(ctx, int(order)))


def xtrg_settn_step(ctx, dtau, order, dev_ptr, nbytes):
    _check(ctx, LIB.xtrg_settn_step(ctx, float(dtau), int(order), C.c_void_p(dev_ptr),
                                    C.c_size_t(nbytes)))


def xtrg_entanglement(ctx, L):
    """MPO entanglement S_E at bonds 1..L-1 (list of L-1 floats)."""
    out = (C.c_double * max(1, L - 1))()
    _check(ctx, LIB.xtrg_entanglement(ctx, out, L - 1))
    return [out[i] for i in range(L - 1)]


def xtrg_checkpoint_bytes(ctx) -> int:
    return int(LIB.xtrg_checkpoint_bytes(ctx))


def xtrg_checkpoint_save(ctx, dev_ptr, nbytes):
    _check(ctx, LIB.xtrg_checkpoint_save(ctx, C.c_void_p(dev_ptr), C.c_size_t(nbytes)))


def xtrg_checkpoint_load(ctx, dev_ptr, nbytes):
    _check(ctx, LIB.xtrg_checkpoint_load(ctx, C.c_void_p(dev_ptr), C.c_size_t(nbytes)))


def xtrg_get_stats(ctx) -> dict:
    o = xtrg_stats()
    _check(ctx, LIB.xtrg_get_stats(ctx, C.byref(o)))
    return o.as_dict()


def xtrg_set_profiling(ctx, on):
    _check(ctx, LIB.xtrg_set_profiling(ctx, 1 if on else 0))


def xtrg_set_graphs(ctx, on):
    _check(ctx, LIB.xtrg_set_graphs(ctx, 1 if on else 0))


def xtrg_set_herm_check(ctx, on):
    _check(ctx, LIB.xtrg_set_herm_check(ctx, 1 if on else 0))


def xtrg_tc_gemm_workspace_bytes(M, N, K, batch, planes, splitk) -> int:
    return int(LIB.xtrg_tc_gemm_workspace_bytes(M, N, K, batch, planes, splitk))


def xtrg_tc_gemm(A_ptr, B_ptr, C_ptr, M, N, K, batch, planes, nprod, splitk, ws_ptr, ws_bytes,
                 stream):
    """Device pointers in, status checked; C = A * B^T per batch (see xtrg.h)."""
    s = LIB.xtrg_tc_gemm(C.c_void_p(A_ptr), C.c_void_p(B_ptr), C.c_void_p(C_ptr), M, N, K, batch,
                         planes, nprod, splitk, C.c_void_p(ws_ptr), C.c_size_t(ws_bytes),
                         C.c_void_p(stream))
    if s != XTRG_OK:
        raise XtrgError(s, "xtrg_tc_gemm")


def xtrg_tc_gemm_nn_workspace_bytes(M, N, K, batch, planes, splitk) -> int:
    return int(LIB.xtrg_tc_gemm_nn_workspace_bytes(M, N, K, batch, planes, splitk))


def xtrg_tc_gemm_nn(A_ptr, B_ptr, C_ptr, M, N, K, batch, planes, nprod, splitk, ws_ptr, ws_bytes,
                    stream):
    """Device pointers in, status checked; C = A * B per batch, B given K x N."""
    s = LIB.xtrg_tc_gemm_nn(C.c_void_p(A_ptr), C.c_void_p(B_ptr), C.c_void_p(C_ptr), M, N, K,
                            batch, planes, nprod, splitk, C.c_void_p(ws_ptr), C.c_size_t(ws_bytes),
                            C.c_void_p(stream))
    if s != XTRG_OK:
        raise XtrgError(s, "xtrg_tc_gemm_nn")


def xtrg_tc_gemm_static(A_ptr, B_ptr, C_ptr, M, N, K, batch, planes, nprod, splitk, stream):
    """xtrg_tc_gemm without a workspace (scratch in a fixed device array);
    returns the status code unchanged so callers can see XTRG_ENOMEM."""
    return int(LIB.xtrg_tc_gemm_static(C.c_void_p(A_ptr), C.c_void_p(B_ptr), C.c_void_p(C_ptr),
                                       M, N, K, batch, planes, nprod, splitk, C.c_void_p(stream)))


def _batch_arrays(Hs, cfgs):
    n = len(Hs)
    if n != len(cfgs) or n == 0:
        raise ValueError("one configuration per Hamiltonian, at least one instance")
    H_arr = (xtrg_mpo * n)(*[h.struct for h in Hs])
    c_arr = (xtrg_config * n)(*cfgs)
    return n, H_arr, c_arr


def xtrg_batch_plan(Hs, cfgs, workspace_bytes, max_concurrent=0):
    """(n_slots, slot_bytes) of a batch in a workspace of the given size."""
    n, H_arr, c_arr = _batch_arrays(Hs, cfgs)
    slots, sb = C.c_int(0), C.c_size_t(0)
    st = LIB.xtrg_batch_plan(n, H_arr, c_arr, workspace_bytes, max_concurrent, C.byref(slots),
                             C.byref(sb))
    if st != XTRG_OK:
        raise XtrgError(st, LIB.xtrg_last_error(None).decode())
    return slots.value, sb.value


def xtrg_batch_run(Hs, cfgs, n_doublings, ws_ptr, ws_bytes, max_concurrent, stream):
    """Rows of observables per instance (list of lists of dicts)."""
    n, H_arr, c_arr = _batch_arrays(Hs, cfgs)
    nd = (C.c_int * n)(*[int(x) for x in n_doublings])
    out = (xtrg_obs * sum(int(x) + 1 for x in n_doublings))()
    st = LIB.xtrg_batch_run(n, H_arr, c_arr, nd, out, ws_ptr, ws_bytes, max_concurrent, stream)
    if st != XTRG_OK:
        raise XtrgError(st, LIB.xtrg_last_error(None).decode())
    rows, k = [], 0
    for x in n_doublings:
        rows.append([out[k + j].as_dict() for j in range(int(x) + 1)])
        k += int(x) + 1
    return rows


def xtrg_last_error(ctx) -> str:
    return LIB.xtrg_last_error(ctx).decode()


def xtrg_destroy(ctx):
    LIB.xtrg_destroy(ctx)
