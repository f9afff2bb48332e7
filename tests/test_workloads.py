"""The seeded workload descriptions: the batched set of 64 chains x 8
interleaved tau0 grids (shape, ranges, determinism) and the small cases."""
import numpy as np

import workloads as wl


def test_batched_instances_shape_and_ranges():
    inst = wl.batched_instances()
    assert len(inst) == 64 * 8
    Ls = {w.L for w in inst}
    assert Ls <= {16, 24, 32, 48, 64}
    assert all(0.0 <= w.Delta <= 1.5 for w in inst)
    assert {w.dstar for w in inst} <= {64, 128, 256}
    for i in range(64):
        grids = inst[8 * i: 8 * i + 8]
        # one chain per group of 8: same L, Delta, D*; tau0 = 2^-12 * 2^(k/8)
        assert len({(w.L, w.Delta, w.dstar) for w in grids}) == 1
        for k, w in enumerate(grids):
            assert abs(w.tau0 - 2.0 ** -12 * 2.0 ** (k / 8)) < 1e-18
            # doubled until beta >= 64, not beyond
            assert w.tau0 * 2 ** w.n_doublings >= 64.0 - 1e-12
            assert w.tau0 * 2 ** (w.n_doublings - 1) < 64.0


def test_batched_instances_are_deterministic():
    a = wl.batched_instances()
    b = wl.batched_instances()
    assert [(w.L, w.Delta, w.dstar) for w in a] == [(w.L, w.Delta, w.dstar) for w in b]
    c = wl.batched_instances(seed=1)
    assert [(w.L, w.Delta) for w in c] != [(w.L, w.Delta) for w in a]


def test_headline_workloads():
    for w in (wl.CHAIN_L64_XX, wl.CHAIN_L64_XXX):
        assert (w.L, w.dstar, w.sweeps, w.tau0) == (64, 256, 4, 2.0 ** -12)
        assert w.betas[-1] == 64.0
    assert wl.CHAIN_L8.betas[-1] == 32.0 and wl.CHAIN_L8.dstar == 256
    assert np.isclose(wl.SQUARE_6X6.tau0 * 2 ** wl.SQUARE_6X6.n_doublings, 32.0)
