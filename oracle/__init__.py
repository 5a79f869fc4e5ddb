"""Oracle: a plain, slow, obviously correct FP64 CPU implementation of the
Improved Seed-CG hot path (Wilson operator, Lanczos with stored basis,
LU-of-T seeding, periodic re-orthogonalisation, CG for the seeded systems).

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only `tests/`, `__graft_entry__.smoke()`
and the `cpu_baseline` / `--impl reference` legs of `bench.py` may import,
call, link or run anything in it.  The CUDA library shares no code with it:
no kernels, headers, helpers, tables or constants.  The only module both
sides use is `paper_0901_3512_gb300.workloads`, which draws seeded inputs
and holds none of the method's arithmetic.

Modules:
  wilson_ref.c / wilson.py  the Wilson-Dirac operator D, D^dag, M = D^dag D
  seedcg.py                 Algorithm 1 (literal), the eq.-(1) Galerkin seed,
                            periodic re-orthogonalisation, CG, classic repeated
                            seeding, Lanczos extremes
  evenodd.py                the even-odd preconditioned (odd-site Schur
                            complement) system of Section 3
  deflation.py              Ritz pairs of T_m and deflated initial guesses
  freefield.py              closed-form free-field spectrum (a pin)
  guess.py                  the learned initial-guess network, forward/backward
  tune_kappa.py             the script that tunes kappa per gauge field
"""
