"""CPU FP64 oracle for the face-based ghost-penalty operator y = G x.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call, link
or execute anything in this package: only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

The oracle computes the plain definition of the operator (Sec. 2.2, ghost
penalty g_F; Sec. 2.4, face matrix entries before factorisation):

    y_I = sum_{F in F_h} sum_{j=1..k} c_j h^{2j-1}
          * integral_F [d_n^j u_x] [d_n^j phi_I] ds,      u_x = sum_J x_J phi_J,

with an explicit dense face matrix per face built from high-order normal
derivatives of the d-dimensional Lagrange basis evaluated at face quadrature
points.  It never uses the Kronecker factorisation of Sec. 2.4 (Eq. for
G_F = M x M x G), shares no code with the CUDA path, and runs in float64.

Modules
  basis         Gauss-Lobatto nodes, Lagrange polynomials in Taylor form,
                Gauss-Legendre rules (numpy.polynomial.legendre)
  mesh          level-set cell classification, ghost-face set, active-DoF
                numbering (lattice-lexicographic, x fastest, compacted)
  ghost_penalty explicit face matrices, y = G x, energy x^T G x, sampled rows
  partition     weighted slab partitions, face owners and DoF windows (Sec. 2.7)

Every function is pinned by the tests in ``tests/test_oracle_*.py`` against
closed forms, brute force and invariants that do not reuse its formulas.
"""
