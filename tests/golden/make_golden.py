"""Write the oracle's thermodynamic rows for the parity workloads.

Calls only ``oracle`` (and the shared ``workloads`` descriptions); no value
here comes from the CUDA path.  Run from the repository root:

    python tests/golden/make_golden.py [name ...]
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


def run(w):
    H = hm.xxz_chain_mpo(w.L, w.J, w.Delta)
    t = time.time()
    rows = xo.run_xtrg(H, w.tau0, w.order, w.dstar, w.sweeps, w.n_doublings,
                       w.svd_rel_tol, init_sweeps=w.init_sweeps)
    return {"workload": w.__dict__, "rows": rows, "oracle_seconds": time.time() - t}


def main(names):
    cases = {w.name: w for w in wl.small_cases() + [wl.CHAIN_L8]}
    for name in names or list(cases):
        out = run(cases[name])
        with open(os.path.join(HERE, f"oracle_{name}.json"), "w") as f:
            json.dump(out, f, indent=1)
        print(name, f"{out['oracle_seconds']:.1f}s")


if __name__ == "__main__":
    main(sys.argv[1:])
