"""FP64 CPU oracle for the truncated SVD of arXiv 2208.08410.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
benchmark's cpu_baseline / reference leg may import, call, link or execute
anything in this package.  The GPU library never uses it and shares no code
with it; the two meet only through the seeded inputs of the synth module.

Modules:
  tsvd_ref  power method, Hotelling and literal deflation, Eq. 1-3, Alg. 4
  philox    Philox-4x32-10 and the Box-Muller start vectors
  jacobi    one-sided Jacobi SVD (brute-force truth for tiny inputs)
  csr_c     plain-C FP64 CSR operator (for sizes NumPy handles slowly)
"""
