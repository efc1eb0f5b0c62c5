"""Paper-like CPU baselines of y = G x, timed beside the oracle by bench.py.

TEST INFRASTRUCTURE ONLY, like ``oracle/``: nothing on the product path imports,
calls, links or executes anything here.  Unlike the oracle, these modules follow
the paper's own method, the tensor-product (Kronecker) factorisation of the face
matrix (Sec. 2.4) applied in one-dimensional steps (Sec. 2.5.1), on the CPU in
FP64; tests/test_baseline_kronecker.py pins them to the oracle.  The oracle never
imports this package.

Modules
  cpu_kronecker  the factorised apply in numpy (BLAS threads) and, through
                 kron_cpu.c (built by build_c.py), in C with OpenMP over faces
"""
