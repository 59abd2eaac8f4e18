"""CPU oracle for the parallel TT-cross quadrature (test infrastructure only).

This package is a plain, slow, obviously correct CPU restatement of what the
GPU path computes, written from the paper (Dolgov & Savostyanov, "Parallel
cross interpolation for high-precision calculation of high-dimensional
integrals", arXiv:1903.11554):

  integrands.py  the Ising-class integrands C_n, D_n, E_n (Sec. 5.1, Eqs. 9-11,
                 and their s-in-R^n form) and the separable TEST family used
                 for the exact-recovery theorem (Thm. 2)
  brute.c/.py    brute-force tensor-product quadrature (Eq. 5) with
                 Neumaier-compensated summation
  exact.py       closed forms and the exact grid value of C_n
  rng.py         the counter-based SplitMix64 draws the cross uses for its
                 random samples (Alg. 2, first step)
  ttcross.py     dimension-parallel greedy cross (Alg. 6 over Alg. 2), QR plus
                 maxvol coefficients (Alg. 1, first step), and the contraction
                 of the weighted cores into the integral (Sec. 4.1)

It is test infrastructure: only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg may import or run anything here.  It shares no code with the
CUDA path; the only common module is the seeded input generator
(paper_1903_11554_gb300.inputs), which holds none of the method's arithmetic.
"""
