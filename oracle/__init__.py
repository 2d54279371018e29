"""CPU FP64 oracle for the interpolative decomposition butterfly factorization (IDBF).

TEST INFRASTRUCTURE ONLY. Nothing in the product package imports this package; only the
tests, the smoke check and the CPU-baseline leg of the benchmark call it. It shares no code
with the CUDA path.

It is a plain, slow restatement of Pang, Ho and Yang, "Interpolative Decomposition Butterfly
Factorization" (arXiv:1809.10573):
  kernels.py  - kernel entries K(x, xi) of the numerical examples (Sec. 3, Examples 1-3)
  sampling.py - Mock-Chebyshev and uniform-random row/column sampling (Sec. 2.1)
  interp.py   - the (eps, k) column and row IDs via a rank-revealing QR (Sec. 2.1, Lemma 2.1)
  idbf.py     - LRCS / MSCS / recursive MSCS construction (Sec. 2.2-2.4), the apply of
                K ~ U^L ... U^h S^h V^h ... V^L (Eq. 1), its adjoint, and the dense matvec
                and sampled relative error used in Sec. 3; on uniform trees (Sec. 2) or on
                coordinate-based dyadic trees with uneven leaves (Sec. 1, Example 3).

Parity pins: every function is checked by tests/test_oracle_*.py against closed forms (DFT),
exact low-rank reconstruction, LAPACK, SVD ranks and brute force on small inputs; the uneven
leaves against an exact rational count, bitwise agreement with the uniform layout on uniform
points, exact reconstruction with empty leaves, and the dense sum of Example 3.
Parity unpinned: none of the functions above.
"""
