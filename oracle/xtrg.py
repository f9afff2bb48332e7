"""Plain CPU XTRG in FP64 (test infrastructure only).

Follows arXiv:1801.00142 step by step, in the order the method states it:

1. rho(tau0) from the series of Eq. RhoTau (Sec. II C), evaluated in Horner
   form; every product H * Y is compressed with the same variational product
   compression as the doubling (App. D.1 names H * X as the typical case), and
   "+ I" is an exact direct sum of MPOs.
2. beta doubling rho_{n+1} = rho_n . rho_n (Eq. rho:scale2, Sec. II B).  The
   product is taken in the positivity-preserving form rho^T rho of Sec. II B
   (rho is real, so the dagger is a transpose of the physical pair); for a
   symmetric rho the two are identical.
3. The product is compressed variationally (App. D.1): minimise
   ||A*B - C||_F^2 (Eq. MPO:prod); with C canonical around sites (i, i+1) the
   stationarity condition Eq. LSEProd gives C_i C_{i+1} = C_E, the generalised
   overlap of Fig. VMPO(a), built from the environments V_L / V_R of
   Fig. VMPO(c).  C_E is split by an SVD (Fig. VMPO(d)): left-to-right the
   left factor takes U and the right factor Lambda V^T; right-to-left Lambda
   goes with U.  Bonds are truncated by *number* (keep D*, Sec. II D), and
   only singular values that are numerically zero are dropped.
4. Normalisation by the Frobenius norm of the orthogonality centre, with the
   log of the scale accumulated, and the thermodynamics of Eq. ThermalQuan.

Tensor convention: an MPO site tensor W[l, s, t, r] is the coefficient of
|s><t| (row spin s, column spin t) between left bond l and right bond r.
The compressed target of ``compress_product(A, B, ...)`` is the operator
A^T B, i.e. (A^T B)_{s,u} = sum_t A_{t,s} B_{t,u}.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from .hamiltonian import identity_mpo


# --------------------------------------------------------------------------
# Environments and the generalised overlap (App. D.1, Fig. VMPO)
# --------------------------------------------------------------------------

def left_env_update(VL, A, B, C):
    """V_L[a,b,c] -> V_L'[a',b',c'] through site tensors A, B, C, in the three
    substeps of Fig. VMPO(c): contract A (cost Da^2 Db Dc d^2), then B over
    (b, t) (cost Da Db^2 Dc d^3), then C over (c, s, u) (cost Da Db Dc^2 d^2)."""
    T = np.tensordot(VL, A, axes=([0], [0]))          # [b, c, t, s, a']
    T = np.tensordot(T, B, axes=([0, 2], [0, 1]))     # [c, s, a', u, b']
    return np.tensordot(T, C, axes=([0, 1, 3], [0, 1, 2]))   # [a', b', c']


def right_env_update(VR, A, B, C):
    """V_R[a',b',c'] -> V_R[a,b,c]: the mirror image of Fig. VMPO(c)."""
    T = np.tensordot(A, VR, axes=([3], [0]))          # [a, t, s, b', c']
    T = np.tensordot(T, B, axes=([1, 3], [1, 3]))     # [a, s, c', b, u]
    return np.tensordot(T, C, axes=([1, 4, 2], [1, 2, 3]))   # [a, b, c]


def left_part(VL, A, B):
    """Left half of Fig. VMPO(a): sum_{a,b,t} V_L[a,b,c] A[a,t,s,a'] B[b,t,u,b'],
    returned as [c, s, u, a', b']."""
    T = np.tensordot(VL, A, axes=([0], [0]))          # [b, c, t, s, a']
    T = np.tensordot(T, B, axes=([0, 2], [0, 1]))     # [c, s, a', u, b']
    return T.transpose(0, 1, 3, 2, 4)


def right_part(A, B, VR):
    """Right half of Fig. VMPO(a): sum_{a'',b'',t'} A[a',t',s',a''] B[b',t',u',b'']
    V_R[a'',b'',c''], returned as [s', u', c'', a', b']."""
    T = np.tensordot(A, VR, axes=([3], [0]))          # [a', t', s', b'', c'']
    T = np.tensordot(T, B, axes=([1, 3], [1, 3]))     # [a', s', c'', b', u']
    return T.transpose(1, 4, 2, 0, 3)


def two_site_overlap(VL, Ai, Bi, Aj, Bj, VR):
    """C_E[c, s, u, s', u', c''] of Eq. LSEProd / Fig. VMPO(a): the target
    A^T B with the holes of C_i C_{i+1} punched at sites (i, i+1)."""
    return np.tensordot(left_part(VL, Ai, Bi), right_part(Aj, Bj, VR),
                        axes=([3, 4], [3, 4]))


# --------------------------------------------------------------------------
# Splitting and canonical form (Fig. VMPO(d))
# --------------------------------------------------------------------------

def kept_count(S, dstar, rel_tol):
    """Number of singular values kept: at most D*, dropping only those at or
    below rel_tol * sigma_max (numerically zero); at least one."""
    if S.size == 0 or S[0] <= 0.0:
        return 1
    k = int(np.count_nonzero(S > rel_tol * S[0]))
    return max(1, min(dstar, k))


def split_two_site(CE, direction, dstar, rel_tol):
    """Split C_E into C_i C_{i+1} by an SVD C_E = U Lambda V^T, keeping the
    largest min(D*, numerical rank) singular values.  direction 'right'
    (left-to-right sweep): C_i = U, C_{i+1} = Lambda V^T.  direction 'left':
    C_i = U Lambda, C_{i+1} = V^T.  Returns (C_i, C_{i+1}, discarded weight)."""
    c, _, _, _, _, z = CE.shape
    M = CE.reshape(c * 4, 4 * z)
    U, S, Vt = np.linalg.svd(M, full_matrices=False)
    k = kept_count(S, dstar, rel_tol)
    tot = float(np.sum(S * S))
    disc = float(np.sum(S[k:] ** 2)) / tot if tot > 0 else 0.0
    if direction == "right":
        Ci = U[:, :k]
        Cj = S[:k, None] * Vt[:k]
    else:
        Ci = U[:, :k] * S[None, :k]
        Cj = Vt[:k]
    return Ci.reshape(c, 2, 2, k), Cj.reshape(k, 2, 2, z), disc, S


def right_canonicalize(C, rel_tol):
    """Bring sites 1..L-1 into right-orthonormal form (rows of each site
    tensor, reshaped l x (s t r), orthonormal), moving the remainder left and
    dropping numerically-zero directions.  The norm ends up in site 0."""
    C = [w.copy() for w in C]
    for i in range(len(C) - 1, 0, -1):
        l, _, _, r = C[i].shape
        M = C[i].reshape(l, 4 * r)
        U, S, Vt = np.linalg.svd(M, full_matrices=False)
        k = kept_count(S, l, rel_tol)
        C[i] = Vt[:k].reshape(k, 2, 2, r)
        C[i - 1] = np.tensordot(C[i - 1], U[:, :k] * S[None, :k], axes=([3], [0]))
    return C


def exact_product(A, B):
    """Exact (fat) MPO of A^T B: fused bonds (a, b), bond dimension Da * Db."""
    out = []
    for a, b in zip(A, B):
        T = np.einsum("atsx,btuy->absuxy", a, b)
        la, lb, _, _, ra, rb = T.shape
        out.append(T.reshape(la * lb, 2, 2, ra * rb))
    return out


@dataclass
class CompressStats:
    max_discarded: float = 0.0
    updates: int = 0
    bond_dims: List[int] = field(default_factory=list)


def compress_product(A, B, guess, dstar, sweeps, rel_tol, stats: Optional[CompressStats] = None):
    """Two-site variational compression of A^T B (App. D.1).

    The guess is right-canonicalised, all right environments are built, then
    ``sweeps`` full sweeps (left-to-right over bonds 0..L-2, then
    right-to-left over bonds L-2..0) solve Eq. LSEProd bond by bond.  On
    return the orthogonality centre is site 0 and sites 1..L-1 are
    right-orthonormal."""
    L = len(A)
    assert L >= 2 and len(B) == L and len(guess) == L
    C = right_canonicalize(guess, rel_tol)
    one = np.ones((1, 1, 1))
    VL = [None] * (L + 1)
    VR = [None] * (L + 1)
    VL[0] = one
    VR[L] = one
    for i in range(L - 1, 0, -1):
        VR[i] = right_env_update(VR[i + 1], A[i], B[i], C[i])
    st = stats if stats is not None else CompressStats()
    for sweep in range(sweeps):
        last = sweep == sweeps - 1
        for i in range(0, L - 1):
            CE = two_site_overlap(VL[i], A[i], B[i], A[i + 1], B[i + 1], VR[i + 2])
            C[i], C[i + 1], disc, _ = split_two_site(CE, "right", dstar, rel_tol)
            VL[i + 1] = left_env_update(VL[i], A[i], B[i], C[i])
            st.updates += 1
            if last:
                st.max_discarded = max(st.max_discarded, disc)
        for i in range(L - 2, -1, -1):
            CE = two_site_overlap(VL[i], A[i], B[i], A[i + 1], B[i + 1], VR[i + 2])
            C[i], C[i + 1], disc, _ = split_two_site(CE, "left", dstar, rel_tol)
            VR[i + 1] = right_env_update(VR[i + 2], A[i + 1], B[i + 1], C[i + 1])
            st.updates += 1
            if last:
                st.max_discarded = max(st.max_discarded, disc)
    st.bond_dims = [w.shape[3] for w in C[:-1]]
    return C


def normalize_center(C):
    """Divide the orthogonality centre (site 0) by its Frobenius norm s;
    with all other sites right-orthonormal, ||C||_F = s.  Returns (C, ln s)."""
    s = float(np.linalg.norm(C[0]))
    C = [w.copy() for w in C]
    C[0] = C[0] / s
    return C, math.log(s)


def direct_sum(P, alpha, Q):
    """Exact MPO of alpha * P + Q by block-diagonal bonds (first site: row
    concatenation, last site: column concatenation)."""
    L = len(P)
    out = []
    for i, (p, q) in enumerate(zip(P, Q)):
        pl, _, _, pr = p.shape
        ql, _, _, qr = q.shape
        if i == 0:
            T = np.zeros((1, 2, 2, pr + qr))
            T[:, :, :, :pr] = alpha * p
            T[:, :, :, pr:] = q
        elif i == L - 1:
            T = np.zeros((pl + ql, 2, 2, 1))
            T[:pl] = p
            T[pl:] = q
        else:
            T = np.zeros((pl + ql, 2, 2, pr + qr))
            T[:pl, :, :, :pr] = p
            T[pl:, :, :, pr:] = q
        out.append(T)
    return out


# --------------------------------------------------------------------------
# Initialisation (Eq. RhoTau) and doubling (Eq. rho:scale2)
# --------------------------------------------------------------------------

def init_rho(H, tau0, order, dstar, sweeps, rel_tol):
    """rho(tau0) = sum_{k=0}^{Nc} (-tau0)^k H^k / k!  (Eq. RhoTau), in Horner
    form Y_{Nc+1} = I, Y_k = I + (-tau0/k) H Y_{k+1}, rho(tau0) = Y_1.  Each
    product H Y (= H^T Y, H real symmetric) is compressed variationally with
    the exact product as the guess.  Returns (normalised rho, ln c) with
    rho(tau0) = e^{ln c} * rho."""
    L = len(H)
    I = identity_mpo(L)
    Y = identity_mpo(L)
    for k in range(order, 0, -1):
        # P = H Y at its true scale (the compression keeps the norm in site 0)
        P = compress_product(H, Y, exact_product(H, Y), dstar, sweeps, rel_tol)
        Y = direct_sum(P, -tau0 / k, I)
    Y = right_canonicalize(Y, rel_tol)
    return normalize_center(Y)


def double(rho, lnc, dstar, sweeps, rel_tol, stats=None):
    """One XTRG step: rho_{n+1} = compress(rho_n^T rho_n), normalised.
    Returns (rho_{n+1}, ln c_{n+1}) with ln c_{n+1} = 2 ln c_n + ln s."""
    C = compress_product(rho, rho, rho, dstar, sweeps, rel_tol, stats)
    C, lns = normalize_center(C)
    return C, 2.0 * lnc + lns


# --------------------------------------------------------------------------
# Traces and thermodynamics (Sec. II B, Eq. ThermalQuan)
# --------------------------------------------------------------------------

def trace(rho):
    """Tr rho by a left-to-right transfer vector."""
    v = np.ones(1)
    for w in rho:
        v = v @ np.trace(w, axis1=1, axis2=2)
    return float(v[0])


def trace_H_rho(H, rho):
    """Tr(H rho) = sum_{s,t} H_{s,t} rho_{t,s}, by a transfer matrix E[h, r]."""
    E = np.ones((1, 1))
    for h, w in zip(H, rho):
        T = np.tensordot(E, h, axes=([0], [0]))            # [r, s, t, h']
        E = np.tensordot(T, w, axes=([0, 1, 2], [0, 2, 1]))  # [h', r']
    return float(E[0, 0])


def trace_H2_rho(H, rho):
    """Tr(H H rho) = sum H_{s,t} H_{t,v} rho_{v,s}, by a transfer tensor E[h1, h2, r]."""
    E = np.ones((1, 1, 1))
    for h, w in zip(H, rho):
        T = np.tensordot(E, h, axes=([0], [0]))            # [h2, r, s, t, h1']
        T = np.tensordot(T, h, axes=([0, 3], [0, 1]))      # [r, s, h1', v, h2']
        E = np.tensordot(T, w, axes=([0, 3, 1], [0, 1, 2]))  # [h1', h2', r']
    return float(E[0, 0, 0])


def frobenius2(rho):
    """||rho||_F^2 = Tr(rho^T rho)."""
    E = np.ones((1, 1))
    for w in rho:
        T = np.tensordot(E, w, axes=([0], [0]))            # [b, s, t, x]
        E = np.tensordot(T, w, axes=([0, 1, 2], [0, 1, 2]))  # [x, y]
    return float(E[0, 0])


def trace_rho_rho(rho):
    """Tr(rho rho) = sum rho_{s,t} rho_{t,s}; equals ||rho||_F^2 iff rho is symmetric."""
    E = np.ones((1, 1))
    for w in rho:
        T = np.tensordot(E, w, axes=([0], [0]))            # [b, s, t, x]
        E = np.tensordot(T, w, axes=([0, 1, 2], [0, 2, 1]))  # [x, y]
    return float(E[0, 0])


def observables(H, rho, lnc, beta, N):
    """Thermodynamics of Eq. ThermalQuan for rho(beta) = e^{lnc} rho:
    ln Z = lnc + ln Tr rho, f = -ln Z/(N beta), u = Tr(H rho)/(N Tr rho),
    c_V = beta^2 (<H^2> - <H>^2)/N; lnZ2 = ln Z(2 beta) = ln ||rho(beta)||_F^2
    (Sec. II B).  herm is the Hermiticity defect ||rho - rho^T||_F / ||rho||_F."""
    tr = trace(rho)
    e1 = trace_H_rho(H, rho) / tr
    e2 = trace_H2_rho(H, rho) / tr
    lnZ = lnc + math.log(tr)
    f2 = frobenius2(rho)
    herm = math.sqrt(max(0.0, 2.0 - 2.0 * trace_rho_rho(rho) / f2))
    return {"beta": beta, "lnZ": lnZ, "f": -lnZ / (N * beta), "u": e1 / N,
            "c": beta * beta * (e2 - e1 * e1) / N, "lnZ2": 2.0 * lnc + math.log(f2),
            "herm": herm}


def run_xtrg(H, tau0, order, dstar, sweeps, n_doublings, rel_tol, init_sweeps=None,
             keep_states=False):
    """Full run: init at beta = tau0, then n_doublings doublings; one row of
    thermodynamics per grid point beta_n = 2^n tau0."""
    L = len(H)
    rho, lnc = init_rho(H, tau0, order, dstar, init_sweeps or sweeps, rel_tol)
    rows = []
    states = []
    beta = tau0
    for n in range(n_doublings + 1):
        if n > 0:
            st = CompressStats()
            rho, lnc = double(rho, lnc, dstar, sweeps, rel_tol, st)
            beta *= 2.0
        row = observables(H, rho, lnc, beta, L)
        row["bond_dims"] = [w.shape[3] for w in rho[:-1]]
        if n > 0:
            row["trunc"] = st.max_discarded
        rows.append(row)
        if keep_states:
            states.append(([w.copy() for w in rho], lnc))
    return (rows, states) if keep_states else rows


def mpo_entanglement(W):
    """MPO entanglement per bond (Sec. IV, Eq. purif): the MPO of rho is read
    as a state with doubled local spaces; at each bond its Schmidt values s_i
    give r_i = s_i^2 / sum s^2 and S_E = -sum r_i ln r_i.  Computed by a
    right-to-left QR pass followed by a left-to-right pass of SVDs of the
    orthogonality centre.  Returns a list of L-1 entropies (bond i between
    sites i and i+1)."""
    W = [w.copy() for w in W]
    L = len(W)
    for i in range(L - 1, 0, -1):
        l, s, t, r = W[i].shape
        Q, R = np.linalg.qr(W[i].reshape(l, s * t * r).T)       # W_i^T = Q R
        W[i] = Q.T.reshape(-1, s, t, r)
        W[i - 1] = np.tensordot(W[i - 1], R.T, axes=([3], [0]))
    out = []
    for i in range(L - 1):
        l, s, t, r = W[i].shape
        U, S, Vt = np.linalg.svd(W[i].reshape(l * s * t, r), full_matrices=False)
        p = S ** 2 / np.sum(S ** 2)
        p = p[p > 0]
        out.append(float(-np.sum(p * np.log(p))))
        W[i] = U.reshape(l, s, t, -1)
        W[i + 1] = np.tensordot(np.diag(S) @ Vt, W[i + 1], axes=([1], [0]))
    return out


# --------------------------------------------------------------------------
# MPO sums (App. D.2, Eq. LSESum) and the pointwise-Taylor SETTN step
# (Sec. II C, Eq. Tay)
# --------------------------------------------------------------------------

def overlap_left_update(VL, T, C):
    """Left environment of the Frobenius overlap <C, T> = sum C_{s,u} T_{s,u}:
    VL[t, c] -> VL'[t', c'] = sum VL[t, c] T[t, s, u, t'] C[c, s, u, c']."""
    X = np.tensordot(VL, T, axes=([0], [0]))              # [c, s, u, t']
    return np.tensordot(X, C, axes=([0, 1, 2], [0, 1, 2]))  # [t', c']


def overlap_right_update(VR, T, C):
    """Right environment: VR[t', c'] -> VR[t, c] = sum T[t, s, u, t'] C[c, s, u, c'] VR[t', c']."""
    X = np.tensordot(T, VR, axes=([3], [0]))              # [t, s, u, c']
    return np.tensordot(X, C, axes=([1, 2, 3], [1, 2, 3]))  # [t, c]


def sum_two_site_overlap(VL, Ti, Tj, VR):
    """C_E of one term of an MPO sum at sites (i, i+1), Fig. VMPO(b): the term
    T with the holes of C_i C_{i+1} punched, [c, s, u, s', u', c'']."""
    X = np.tensordot(VL, Ti, axes=([0], [0]))             # [c, s, u, t']
    X = np.tensordot(X, Tj, axes=([3], [0]))              # [c, s, u, s', u', t'']
    return np.tensordot(X, VR, axes=([5], [0]))           # [c, s, u, s', u', c'']


def compress_sum(terms, weights, guess, dstar, sweeps, rel_tol, stats=None):
    """Two-site variational compression of sum_j w_j T_j (App. D.2): minimise
    ||sum_j w_j T_j - C||_F^2 (Eq. MPO:plus); with C canonical around sites
    (i, i+1) the stationarity condition Eq. LSEProd's sum analogue (Eq.
    LSESum) gives C_i C_{i+1} = sum_j w_j C_{E,j}, split as in the product
    compression.  Returns C with its orthogonality centre at site 0."""
    L = len(guess)
    n = len(terms)
    assert n == len(weights) and all(len(t) == L for t in terms)
    C = right_canonicalize(guess, rel_tol)
    one = np.ones((1, 1))
    VL = [[None] * (L + 1) for _ in range(n)]
    VR = [[None] * (L + 1) for _ in range(n)]
    for j in range(n):
        VL[j][0] = one
        VR[j][L] = one
        for i in range(L - 1, 0, -1):
            VR[j][i] = overlap_right_update(VR[j][i + 1], terms[j][i], C[i])
    st = stats if stats is not None else CompressStats()

    def ce(i):
        return sum(w * sum_two_site_overlap(VL[j][i], terms[j][i], terms[j][i + 1], VR[j][i + 2])
                   for j, w in enumerate(weights))

    for sweep in range(sweeps):
        last = sweep == sweeps - 1
        for i in range(0, L - 1):
            C[i], C[i + 1], disc, _ = split_two_site(ce(i), "right", dstar, rel_tol)
            for j in range(n):
                VL[j][i + 1] = overlap_left_update(VL[j][i], terms[j][i], C[i])
            st.updates += 1
            if last:
                st.max_discarded = max(st.max_discarded, disc)
        for i in range(L - 2, -1, -1):
            C[i], C[i + 1], disc, _ = split_two_site(ce(i), "left", dstar, rel_tol)
            for j in range(n):
                VR[j][i + 1] = overlap_right_update(VR[j][i + 2], terms[j][i + 1], C[i + 1])
            st.updates += 1
            if last:
                st.max_discarded = max(st.max_discarded, disc)
    st.bond_dims = [w.shape[3] for w in C[:-1]]
    return C


def settn_step(H, rho, lnc, dtau, order, dstar, sweeps, rel_tol, stats=None):
    """One pointwise-Taylor step of SETTN (Eq. Tay, Fig. SETTNAlg(b)):
    rho(tau + dtau) = sum_{k=0}^{order} (-dtau)^k / k! H^k rho(tau), with
    rho(tau) = e^{lnc} rho.  The terms H^k rho are built one from the other by
    compressed products H (H^{k-1} rho) (App. D.1, guess: the previous term),
    and their weighted sum by the variational MPO sum (App. D.2, guess: rho).
    Returns the normalised result and its ln c."""
    terms = [rho]
    for _ in range(order):
        prev = terms[-1]
        terms.append(compress_product(H, prev, prev, dstar, sweeps, rel_tol))
    weights = [(-dtau) ** k / math.factorial(k) for k in range(order + 1)]
    C = compress_sum(terms, weights, rho, dstar, sweeps, rel_tol, stats)
    C, lns = normalize_center(C)
    return C, lnc + lns


def run_settn(H, tau0, init_order, dstar, sweeps, n_steps, taylor_order, rel_tol):
    """SETTN on the logarithmic grid tau_n = 2^n tau0: the series
    initialisation of Eq. RhoTau, then pointwise-Taylor steps tau_n ->
    tau_{n+1} = 2 tau_n (Eq. Tay, dtau = tau_n).  One row of thermodynamics
    per grid point, as run_xtrg."""
    L = len(H)
    rho, lnc = init_rho(H, tau0, init_order, dstar, sweeps, rel_tol)
    beta = tau0
    rows = []
    for n in range(n_steps + 1):
        if n > 0:
            st = CompressStats()
            rho, lnc = settn_step(H, rho, lnc, beta, taylor_order, dstar, sweeps, rel_tol, st)
            beta *= 2.0
        row = observables(H, rho, lnc, beta, L)
        row["bond_dims"] = [w.shape[3] for w in rho[:-1]]
        if n > 0:
            row["trunc"] = st.max_discarded
        rows.append(row)
    return rows


def expectation(O, rho):
    """<O> = Tr(O rho) / Tr rho for an operator MPO O (the transfer of
    trace_H_rho with O in place of H)."""
    return trace_H_rho(O, rho) / trace(rho)


def binder_ratio(M2, M4, rho):
    """U_4 = <M^2>^2 / <M^4> (Sec. IV D, Eq. Binder) from the MPOs of
    (S^z_tot)^2 and (S^z_tot)^4."""
    m2 = expectation(M2, rho)
    return m2 * m2 / expectation(M4, rho)
