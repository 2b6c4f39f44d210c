"""Eigenvalue sensitivity to the per-element damping coefficients (oracle).

Plain FP64 restatement, test infrastructure only.  The paper has no
sensitivity analysis; the formula is the first-order perturbation of a simple
eigenvalue of the QEP (K + lambda C + lambda^2 M) x = 0 of Eq. (QuadEig).
K, M, C are real symmetric, so the left eigenvector is the unconjugated x and
for C = sum_e sigma_e M_e:

  d lambda / d sigma_e = - lambda (x_e^T M_e x_e) / (x^T (2 lambda M + C) x),

x_e being the restriction of x to the DOFs of element e (transpose, not
conjugate transpose).
"""
import numpy as np

from .bspline import Space1D


def element_quadratic_forms(ne, p, block, x, nq=None):
    """q_e = x_e^T M_e x_e for every element e = ex + ne*ey (complex x).

    M_e is recomputed here from its Gauss-quadrature definition (same points
    and weights as the assembly) and applied to the element's DOFs; Dirichlet
    functions carry no DOF and contribute zero.
    """
    nq = p + 1 if nq is None else nq
    sp1 = Space1D(ne, p, block)
    n, nf = sp1.n, sp1.n_full
    tabs = sp1.element_tables(nq)
    x = np.asarray(x).reshape(n, n)           # [iy, ix]
    out = np.zeros(ne * ne, dtype=np.result_type(x, np.float64))
    for ey in range(ne):
        iy, vy, _, wy = tabs[ey]
        for ex in range(ne):
            ix, vx, _, wx = tabs[ex]
            # element mass matrix, 2-D quadrature over the nq x nq points
            B = np.einsum('qa,rb->qrab', vx, vy)
            W = np.outer(wx, wy)
            Me = np.einsum('qr,qrab,qrcd->abcd', W, B, B)
            xe = np.zeros((len(ix), len(iy)), dtype=out.dtype)
            for a, gx in enumerate(ix):
                for b, gy in enumerate(iy):
                    if 1 <= gx <= nf - 2 and 1 <= gy <= nf - 2:
                        xe[a, b] = x[gy - 1, gx - 1]
            out[ex + ne * ey] = np.einsum('ab,abcd,cd->', xe, Me, xe)
    return out


def damping_gradient(ne, p, block, lam, X, C, M, nq=None):
    """G[k, e] = d lambda_k / d sigma_e for eigenpairs (lam[k], X[k])."""
    G = []
    for lk, xk in zip(lam, X):
        qe = element_quadratic_forms(ne, p, block, xk, nq)
        den = xk @ (2.0 * lk * (M @ xk) + C @ xk)
        G.append(-lk * qe / den)
    return np.array(G)
