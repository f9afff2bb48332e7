"""CPU checks of the C ABI: the library loads and exports every function the
header declares, and the host-side argument checks reject bad input without
touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "xtrg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(xtrg_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1801_00142_gb300.build import build
    build()
    from paper_1801_00142_gb300 import _lib
    return _lib


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 11
    so = ctypes.CDLL(lib.LIB_PATH)
    for n in names:
        assert hasattr(so, n), n
    assert sorted(lib.SYMBOLS) == names


def test_workspace_bytes_and_input_checks(lib):
    from paper_1801_00142_gb300.hamiltonians import xxz_chain
    dims, sites = xxz_chain(8)
    H = lib.MpoArgs(dims, sites)
    cfg = lib.make_config(2 ** -10, 4, 256, 4)
    n = lib.xtrg_workspace_bytes(H, cfg)
    assert n > 0
    # larger D* needs more memory; bad configs give 0 bytes
    assert lib.xtrg_workspace_bytes(H, lib.make_config(2 ** -10, 4, 512, 4)) > n
    assert lib.xtrg_workspace_bytes(H, lib.make_config(2 ** -10, 4, 0, 4)) == 0
    # the orthonormalisation block width: 0 (default) or 32..256 in steps of 32
    for ob in (32, 96, 256):
        assert lib.xtrg_workspace_bytes(H, lib.make_config(2 ** -10, 4, 256, 4, prec="bf16x6",
                                                           orth_block=ob)) > 0
    for ob in (-32, 16, 48, 288):
        assert lib.xtrg_workspace_bytes(H, lib.make_config(2 ** -10, 4, 256, 4, prec="bf16x6",
                                                           orth_block=ob)) == 0
    bad = lib.MpoArgs([2] + dims[1:], sites)
    assert lib.xtrg_workspace_bytes(bad, cfg) == 0
    # create rejects a NULL workspace before any device call
    with pytest.raises(lib.XtrgError) as e:
        lib.xtrg_create(H, cfg, 0, n, 0)
    assert e.value.status == lib.XTRG_EINVAL
    # and a workspace that is too small
    with pytest.raises(lib.XtrgError) as e:
        lib.xtrg_create(H, cfg, 256, n - 1024, 0)
    assert e.value.status == lib.XTRG_ENOMEM


@pytest.mark.parametrize("L,dstar,prec", [(2, 1, "fp64"), (4, 16, "fp64"), (8, 256, "fp64"),
                                          (64, 256, "fp64"), (10, 3, "fp64"), (8, 256, "bf16x6"),
                                          (64, 256, "bf16x6"), (10, 320, "bf16x6"),
                                          (12, 1024, "bf16x3")])
def test_workspace_plan_covers_every_buffer(lib, L, dstar, prec):
    """With exactly xtrg_workspace_bytes() the carving of every buffer fits:
    on a machine without a GPU, create then fails at its first device copy
    (XTRG_ECUDA), never at carving (XTRG_ENOMEM)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("host-only check")
    from paper_1801_00142_gb300.hamiltonians import xxz_chain
    dims, sites = xxz_chain(L)
    H = lib.MpoArgs(dims, sites)
    cfg = lib.make_config(2 ** -10, 4, dstar, 2, prec=prec)
    n = lib.xtrg_workspace_bytes(H, cfg)
    with pytest.raises(lib.XtrgError) as e:
        lib.xtrg_create(H, cfg, 1 << 20, n, 0)
    assert e.value.status == lib.XTRG_ECUDA


def test_hamiltonian_builder_is_the_xxz_chain(lib):
    import numpy as np

    from oracle import hamiltonian as oh
    from paper_1801_00142_gb300.hamiltonians import xxz_chain
    for L, D in ((2, 1.0), (5, 0.35), (7, 1.3)):
        dims, sites = xxz_chain(L, 1.0, D)
        assert dims[0] == dims[-1] == 1 and all(d == 5 for d in dims[1:-1])
        assert np.abs(oh.mpo_to_dense(sites) - oh.dense_xxz(L, 1.0, D)).max() < 1e-14


def test_context_calls_reject_a_null_context(lib):
    """Every entry point that takes a context returns XTRG_EINVAL for NULL
    before touching the device (the switches, the state and stats calls)."""
    L = lib.LIB
    assert L.xtrg_set_graphs(None, 1) == lib.XTRG_EINVAL
    assert L.xtrg_set_herm_check(None, 0) == lib.XTRG_EINVAL
    assert L.xtrg_set_profiling(None, 1) == lib.XTRG_EINVAL
    assert L.xtrg_init(None) == lib.XTRG_EINVAL
    assert L.xtrg_double(None) == lib.XTRG_EINVAL
    st = lib.xtrg_stats()
    assert L.xtrg_get_stats(None, ctypes.byref(st)) == lib.XTRG_EINVAL
