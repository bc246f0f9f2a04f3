"""Plain FP64 CPU oracle for the control equation of the tensor method.

TEST INFRASTRUCTURE ONLY. Only the test suite (tests/), the smoke check in
__graft_entry__.smoke() and the CPU-baseline leg of bench.py may import, call
or execute anything in this package. The GPU library never uses it, and it
never uses the GPU library: the two share no code. Both are fed by the seeded
input generator paper_2006_09314_gb300.inputs, which holds none of the
method's arithmetic.

What the oracle computes (NumPy + SciPy LAPACK, float64, no blocking or fusion
beyond what each definition states):

  operator.py   Section 3.2 (1D finite-difference Sturm-Liouville matrices),
                Section 3.3 (eigen-decomposition A_l = V_l diag(lambda) V_l^T,
                Kronecker-sum structure), the 7-point stencil of A and the
                dense Kronecker sum (for pins).
  fullgrid.py   Sections 3.3-3.4: the exact discrete control solve
                u* = (xV) [((xV^T) y) ./ F2(lambda_i+lambda_j+lambda_k)] by
                full-grid diagonalization, F(A)x for any spectral function,
                and a slab-streamed relative error for grids that do not fit.
  formats.py    Appendix 1: canonical and Tucker tensors by definition
                (expansion, Euclidean inner product, Hadamard product, sums).
  expsum.py     Section 3.4 (Laplace transform + sinc quadrature of s^-alpha
                and of s^(alpha-1), Hadamard split D^alpha = D * D^(alpha-1));
                the preconditioner spectral function (Section 3.5, case (B)).
  truncation.py Appendix 1: canonical-to-Tucker by reduced HOSVD, Tucker core
                truncation and Tucker-to-canonical (the `trunc` procedure).
  pcg.py        Appendix 2, Algorithm 1: preconditioned CG in low-rank format.

Every function is pinned by the tests in tests/test_oracle_*.py against
closed forms, brute force on tiny grids, invariants or special cases the
paper names; none of its expected values comes from the GPU path.
"""
