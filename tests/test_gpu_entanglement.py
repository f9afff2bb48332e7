"""GPU parity of the MPO entanglement S_E (Sec. IV A, Eq. purif) through the C
ABI (xtrg_entanglement) against the oracle's mpo_entanglement, which is
pinned on the dense operator Schmidt decomposition.  Both act on the same
state (the GPU's rho, read back through xtrg_get_state), so the comparison
is of the entanglement computation alone: FP64 on both sides."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng_cls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_00142_gb300.build import build
    build()
    from paper_1801_00142_gb300.engine import XTRG
    return XTRG


def _check(eng, L, n_doublings):
    from oracle import xtrg as ox
    eng.init()
    worst = 0.0
    for n in range(n_doublings + 1):
        if n:
            eng.double()
        S = eng.entanglement()
        sites, lnc, beta = eng.get_state()
        ref = ox.mpo_entanglement(sites)
        assert len(S) == L - 1
        d = max(abs(a - b) for a, b in zip(S, ref))
        worst = max(worst, d)
        assert d <= 1e-10 * max(1.0, max(ref)), (beta, S, ref)
        # the state itself is unchanged by the measurement
        s2, lnc2, beta2 = eng.get_state()
        assert lnc2 == lnc and beta2 == beta
        assert all(np.array_equal(a, b) for a, b in zip(sites, s2))
    return worst, S


def test_entanglement_of_a_chain_matches_oracle(eng_cls):
    L = 8
    eng = eng_cls.xxz(L, 1.0, 1.0, tau0=2.0 ** -6, dstar=64, sweeps=2)
    worst, S = _check(eng, L, 8)
    print("max |dS|", worst, "S(beta=4)", S)
    # as beta -> 0, rho -> identity, a product operator: S_E = O(beta^2 ln(1/beta))
    e0 = eng_cls.xxz(L, 1.0, 1.0, tau0=2.0 ** -10, dstar=64, sweeps=2)
    e0.init()
    assert max(e0.entanglement()) < 1e-4
    # reflection symmetry of the open chain
    assert abs(S[0] - S[-1]) < 1e-8 and abs(S[2] - S[-3]) < 1e-8


def test_entanglement_of_a_snake_lattice_matches_oracle(eng_cls):
    import workloads as wl
    bonds = wl.square_snake_bonds(2, 3)
    eng = eng_cls.from_bonds(6, bonds, tau0=2.0 ** -6, dstar=64, sweeps=2)
    worst, S = _check(eng, 6, 6)
    print("snake max |dS|", worst, S)


def test_entanglement_after_mixed_doublings_and_from_a_general_gauge(eng_cls):
    """After tensor-core doublings (state in right-canonical form) and after
    set_state of the same MPO in an arbitrary gauge (re-canonicalised inside
    the call), the entropies agree with the oracle on that state."""
    from oracle import xtrg as ox
    L = 8
    eng = eng_cls.xxz(L, 1.0, 0.5, tau0=2.0 ** -6, dstar=32, sweeps=2, prec="bf16x6")
    eng.init()
    for _ in range(6):
        eng.double()
    S = eng.entanglement()
    sites, lnc, beta = eng.get_state()
    ref = ox.mpo_entanglement(sites)
    assert max(abs(a - b) for a, b in zip(S, ref)) <= 1e-10
    # scramble the gauge: insert G G^-1 on every bond
    rng = np.random.default_rng(3)
    g = [w.copy() for w in sites]
    for i in range(L - 1):
        D = g[i].shape[3]
        G = np.eye(D) + 0.3 * rng.standard_normal((D, D))
        g[i] = np.tensordot(g[i], G, axes=([3], [0]))
        g[i + 1] = np.tensordot(np.linalg.inv(G), g[i + 1], axes=([1], [0]))
    eng.set_state(g, lnc, beta, right_canonical=False)
    S2 = eng.entanglement()
    assert max(abs(a - b) for a, b in zip(S2, ref)) <= 1e-9
