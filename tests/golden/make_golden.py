"""Write the oracle's thermodynamic rows for the parity workloads.

Calls only ``oracle`` (and the shared ``workloads`` descriptions); no value
here comes from the CUDA path.  Run from the repository root:

    python tests/golden/make_golden.py [name ...]
    python tests/golden/make_golden.py --long xx_L32_D256

``--long`` runs one of the long FP64 reference schedules row by row and
rewrites its file after every doubling (hours of CPU at D* = 256; no
perturbation sensitivity is computed for these).
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402
from oracle import hamiltonian as hm  # noqa: E402
from oracle import xtrg as xo  # noqa: E402


def _run(w, H):
    return xo.run_xtrg(H, w.tau0, w.order, w.dstar, w.sweeps, w.n_doublings,
                       w.svd_rel_tol, init_sweeps=_init_sweeps(w))


def hamiltonian(w):
    """The oracle's MPO of a workload: the chain automaton, or for a lattice
    the distance automaton of its snake bond list."""
    if isinstance(w, wl.LatticeWorkload):
        return hm.bonds_mpo(w.N, w.bonds())
    return hm.xxz_chain_mpo(w.L, w.J, w.Delta)


def _init_sweeps(w):
    return getattr(w, "init_sweeps", None) or w.sweeps


def run(w):
    """Oracle rows; for truncated runs also the oracle's own sensitivity: the
    largest change of each row over three seeded perturbations of the
    nonzero entries of H by 1e-14 relative noise (several truncated results are equally optimal when
    D* cuts through a degenerate set of singular values, so a parity bar
    below this sensitivity would be meaningless)."""
    import numpy as np
    H = hamiltonian(w)
    t = time.time()
    rows = _run(w, H)
    secs = time.time() - t
    truncated = any(r.get("trunc", 0.0) > 1e-24 for r in rows)
    if truncated:
        for r in rows:
            r["sens"] = {"lnZ": 0.0, "u": 0.0, "c": 0.0}
        for seed in (7, 8, 9):
            rng = np.random.default_rng(seed)
            Hp = [h * (1.0 + 1e-14 * rng.standard_normal(h.shape)) for h in H]
            pert = _run(w, Hp)
            for r, q in zip(rows, pert):
                for k in ("lnZ", "u", "c"):
                    r["sens"][k] = max(r["sens"][k], abs(r[k] - q[k]))
    return {"workload": w.__dict__, "rows": rows, "oracle_seconds": secs,
            "truncated": truncated}


def run_long(w, path):
    """Init, then the doublings one at a time, writing the rows so far after
    each (so a long run can be followed and is not lost if interrupted)."""
    H = hamiltonian(w)
    t0 = time.time()
    rho, lnc = xo.init_rho(H, w.tau0, w.order, w.dstar, _init_sweeps(w), w.svd_rel_tol)
    beta = w.tau0
    rows = []
    for n in range(w.n_doublings + 1):
        if n > 0:
            st = xo.CompressStats()
            rho, lnc = xo.double(rho, lnc, w.dstar, w.sweeps, w.svd_rel_tol, st)
            beta *= 2.0
        row = xo.observables(H, rho, lnc, beta, w.L)
        row["bond_dims"] = [x.shape[3] for x in rho[:-1]]
        if n > 0:
            row["trunc"] = st.max_discarded
        row["elapsed_s"] = time.time() - t0
        rows.append(row)
        with open(path + ".tmp", "w") as f:
            json.dump({"workload": w.__dict__, "rows": rows, "oracle_seconds": time.time() - t0,
                       "truncated": any(r.get("trunc", 0.0) > 1e-24 for r in rows),
                       "complete": n == w.n_doublings}, f, indent=1)
        os.replace(path + ".tmp", path)
        print(w.name, f"beta={beta:g}", f"{time.time() - t0:.0f}s", flush=True)


def main(names):
    cases = {w.name: w for w in wl.small_cases() + [wl.CHAIN_L8] + wl.small_lattice_cases()}
    for name in names or list(cases):
        out = run(cases[name])
        with open(os.path.join(HERE, f"oracle_{name}.json"), "w") as f:
            json.dump(out, f, indent=1)
        print(name, f"{out['oracle_seconds']:.1f}s")


LONG = {w.name: w for w in (wl.CHAIN_L32_XX, wl.CHAIN_L64_XX)}

if __name__ == "__main__":
    if sys.argv[1:2] == ["--long"]:
        for name in sys.argv[2:]:
            run_long(LONG[name], os.path.join(HERE, f"oracle_{name}.json"))
    else:
        main(sys.argv[1:])
