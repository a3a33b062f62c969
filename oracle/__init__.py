"""FP64 CPU oracle for the level-set / adjoint LLG hot path.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this package: only the tests, the smoke check and the CPU-baseline
leg of the benchmark use it.  It shares no code with the CUDA library; the
only module both sides read is the seeded input generator `workloads`.

Each function is a plain, slow restatement of the discrete method:
  demag.py     cell-averaged demagnetising tensor (Newell, Williams and Dunlop
               1993 closed form near the origin, Gauss quadrature of the
               dipole kernel far from it), direct O(N^2) demag sum and the
               zero-padded FFT convolution.
  llg.py       material map (Eq. 4), effective field, LL right-hand side of
               Eq. 11, classic RK4, objectives (Eq. 9 size term, Eq. 10-style
               port functional), the exact discrete adjoint of RK4 (Eq. 6/7 in
               discrete form) and the level-set step (Eq. 5 with the
               renormalisation of the Results section).
  schedule.py  checkpoint schedules for the reverse sweep.
"""
