"""Plain FP64 CPU oracle for the rIGA shift-and-invert QEP solve.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference leg may import or run this package;
the library path never does, and it shares no code with the CUDA path.

Modules (each cites the part of the paper it restates):
  bspline      knots, Cox--de Boor values/derivatives, C^0 separator functions
  pattern      H(curl)/H^1 matrix sizes and pattern counts (Fig. 4 sizes)
  assemble     Gauss-quadrature Galerkin K, M and C = sum_e sigma_e M_e
  nd           separator-induced nested dissection + supernodal symbolic phase
  multifrontal multifrontal LDL^T of Q(s) and supernodal FB solves
  qep          block operator, B-inner product, CGS2 Arnoldi, Krylov--Schur,
               Ritz values, eigenvectors and backward errors
  adjoint      d lambda / d sigma_e

Pins (tests/test_oracle_pins.py): scipy's independent B-splines, the paper's
printed Fig. 4 sizes, tensor-product identities of M and K, brute-force
symbolic elimination, dense LDL^T reconstruction, the dense 2N pencil,
LAPACK QZ eigenvalues, the proportional-damping closed form, the undamped
limit, a gradient sum rule and central differences.
"""
