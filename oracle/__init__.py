"""FP64 CPU oracle for the ADMM QP solver (TEST INFRASTRUCTURE ONLY).

This package is a plain, slow, direct restatement of the paper's method
(Schubiger, Banjac, Lygeros, "GPU Acceleration of ADMM for Large-Scale
Quadratic Programming"), used to check the GPU solver.  Only the tests, the
package-level ``smoke()`` check and the CPU-baseline and reference legs of
``bench.py`` may import it.  It shares no code with the GPU path: no kernels, headers,
helpers, constants or pre/post-processing.  The GPU path must never import,
load or call anything here.

Modules:
  ldl.c / ldl.py  sparse LDL' of the quasi-definite KKT matrix (Section 3.2)
  schur.c / dense.py  dense Cholesky of the KKT matrix's Schur complement on
                  the variables (the reduced system of eq. (kkt_red_sc)), for
                  problems with few variables and many constraints
  admm.py         Ruiz equilibration (Algorithm 2), ADMM (Algorithm 1) with
                  the direct KKT solve, PCG (Algorithm 3) on the reduced KKT
                  system (Section 5.3), residuals and tolerances (Section 3.1),
                  infeasibility certificates (Section 3.1), the Jacobi
                  preconditioner (scalar R or the rho vector of eq. (rho_vec)),
                  rho adaptation
  checks.py       solution checks that do not run ADMM: the optimality
                  conditions (Section 2.1), brute-force active sets, the
                  closed-form box QP, the duality gap
  formats.py      COO / CSR / CSC conversions of Section 4.3
  mlp.py          FP64 forward / backward / Adam for the rho-policy MLP
                  (parity unpinned against the paper: the paper has no MLP;
                  pinned by finite differences and a hand-built network)
  policy.py       the learned rho decision and its stall rule, restated from
                  the solver's readings (parity unpinned against the paper;
                  pinned by hand-built networks and a hand-traced stall
                  sequence)
"""
