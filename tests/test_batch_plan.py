"""Host-side checks of the batch runner's planning (no GPU): slot size = the
largest instance's workspace rounded up to 256 bytes, slot count bounded by
the instances, the concurrency cap and the workspace; errors are reported
through xtrg_last_error(NULL); without a device the run fails cleanly."""
import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_1801_00142_gb300.build import build
    build()
    from paper_1801_00142_gb300 import _lib
    return _lib


def _instances(lib):
    from paper_1801_00142_gb300.hamiltonians import xxz_chain
    out = []
    for L, D in ((8, 16), (16, 64), (12, 32)):
        dims, sites = xxz_chain(L)
        out.append((lib.MpoArgs(dims, sites), lib.make_config(2 ** -10, 4, D, 2, prec="bf16x6")))
    return [h for h, _ in out], [c for _, c in out]


def test_plan_slot_size_and_count(lib):
    Hs, cfgs = _instances(lib)
    need = max(-(-lib.xtrg_workspace_bytes(h, c) // 256) * 256 for h, c in zip(Hs, cfgs))
    slots, sb = lib.xtrg_batch_plan(Hs, cfgs, 100 * need, 0)
    assert sb == need and slots == 3                 # bounded by the 3 instances
    assert lib.xtrg_batch_plan(Hs, cfgs, 100 * need, 2)[0] == 2      # concurrency cap
    assert lib.xtrg_batch_plan(Hs, cfgs, 2 * need + need // 2, 0)[0] == 2   # workspace


def test_plan_errors(lib):
    Hs, cfgs = _instances(lib)
    need = max(lib.xtrg_workspace_bytes(h, c) for h, c in zip(Hs, cfgs))
    with pytest.raises(lib.XtrgError) as e:
        lib.xtrg_batch_plan(Hs, cfgs, need // 2, 0)
    assert e.value.status == lib.XTRG_ENOMEM and "holds no instance" in str(e.value)
    bad = list(cfgs)
    bad[1] = lib.make_config(2 ** -10, 4, 0, 2)      # D* = 0 is invalid
    with pytest.raises(lib.XtrgError) as e:
        lib.xtrg_batch_plan(Hs, bad, 1 << 40, 0)
    assert e.value.status == lib.XTRG_EINVAL and "instance 1" in str(e.value)


def test_run_without_device_fails_cleanly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    Hs, cfgs = _instances(lib)
    with pytest.raises(lib.XtrgError) as e:
        lib.xtrg_batch_run(Hs, cfgs, [2, 2, 2], 1 << 20, 1 << 40, 0, None)
    assert e.value.status == lib.XTRG_ECUDA
    with pytest.raises(lib.XtrgError) as e:                      # misaligned workspace
        lib.xtrg_batch_run(Hs, cfgs, [2, 2, 2], (1 << 20) + 8, 1 << 40, 0, None)
    assert e.value.status == lib.XTRG_EINVAL
