"""FP64 CPU oracle for the double-grid interpolated BSE Haydock path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only the test suite, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may use it.  It shares no code with the CUDA library; the only
common input is `paper_1602_01863_gb300.synth`, which draws the seeded model
parameters and holds none of the method's arithmetic.

Modules
  model    grids, trilinear weights, the synthetic model crystal, the explicit
           kernel (Sec. 2, Eqs. bse1-bse3b) and K_c on the coarse mesh
  interp   band overlaps d (Eq. completeness), the interpolation operator F
           (Eqs. interpwfn, interp1), M1 and M3 (Sec. 4) in dense and
           matrix-free (Eqs. matmul1-matmul3) form
  haydock  Lanczos recursion (Eqs. ai, bi, ci), continued fraction
           (Eq. fraccont) and brute-force diagonalisation

Everything is complex128 / float64 and written for clarity, not speed.
"""
