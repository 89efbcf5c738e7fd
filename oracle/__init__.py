"""Plain, slow CPU oracle for the matrix-free hexahedral mass/diffusion action.

TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library and its
Python binding) may import, call or link this package; only the tests, the
smoke check in ``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` do.

What it computes is the plain definition of the discrete operator the paper
factors (Section 2, the operator-level form A_L = block-diag(A^e) with
A^e = D^T G^e D): for every element, the quadrature sum

    y^e_i = sum_q  grad(phi_i)(x_q) . K_q grad(phi_j)(x_q) |det J_q| w_q  u^e_j

evaluated densely, with basis functions tabulated directly at every 3D
quadrature point (no sum factorization, no 1D contraction passes), followed by
a scatter-add in fixed element order.  Sum factorization (Section 1, the
O(p^{2d}) -> O(p^{d+1}) reduction) is an exact reordering of these same sums,
so a fused GPU kernel must reproduce this result up to rounding order.

Modules:
  quadrature  Gauss / Gauss-Lobatto rules (Newton on Legendre polynomials),
              Lagrange basis values and derivatives by the product formula.
  fem         trilinear geometry, quadrature data by definition, dense element
              action, assembled sparse matrix (tiny meshes), Dirichlet masking,
              Jacobi diagonal, preconditioned CG, manufactured right-hand side,
              L2 error, and the adjoint gradient of 0.5 ||A(k) x - b||^2.

Every function is pinned by a ``-m "not gpu"`` test against something other
than itself (closed forms, library routines, invariants, brute force); see the
tests named test_oracle_*.py.
"""
