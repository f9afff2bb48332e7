"""FP64 CPU oracle for the XTRG doubling path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only the tests, the smoke check and the CPU-baseline leg
of the benchmark use it.  It shares no code with the CUDA path; the only module
both sides import is ``workloads`` (seeded workload descriptions, no method
arithmetic).

Contents (each function cites the passage of arXiv:1801.00142 it follows):

* ``hamiltonian``  dense XXZ Hamiltonians and the automaton MPO of App. B.1
* ``exact``        exact diagonalisation thermodynamics (the paper's ED
                   reference), the free-fermion closed form of App. F for the
                   XY chain, and the two-site closed form
* ``xtrg``         a plain, step-by-step CPU XTRG: series initialisation
                   (Eq. RhoTau), beta doubling (Eq. rho:scale2) by the two-site
                   variational product compression of App. D.1 (Eq. LSEProd,
                   Fig. VMPO), normalisation, and the thermodynamic quantities
                   of Eq. ThermalQuan

Everything is numpy in float64.  Pins (tests that tie the oracle to something
other than itself) live in ``tests/test_oracle_*.py``.
"""
