"""FP64 CPU oracle for the parallel step-wise pulling protocol.

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py are the only callers.  Nothing here
imports the CUDA package and the CUDA package never imports this one; both
consume only the seeded inputs of paper_1105_4840_gb300.inputs.

Contents
  _clib.py        ctypes binding of oracle.c (Philox, chain energy / forces,
                  BAOAB and overdamped Langevin runs)
  estimators.py   Eq. (9) work, Eq. (12) JE, Eq. (13) Gaussian, Eq. (14)
                  alternative formula, combined estimate, jackknife errors,
                  Zuckerman-Woolf variance
  quadrature.py   exact F(lambda, k) by quadrature for the 1D model and the
                  Gaussian chain
  build.py        compiles oracle.c with gcc
"""
