"""Galerkin matrices K, M and C of the scalar model problem (oracle).

Plain FP64 restatement, test infrastructure only.

Space: tensor-product B-splines B_{ij} = N_i(xi) N_j(eta) (Section 3.1) on the
unit square with the identity geometric map, IGA or rIGA knots (Sections
3.2--3.3), homogeneous Dirichlet functions removed.  DOF id = i + n*j with the
xi index i fastest; element id = ex + ne*ey.

Matrices (scalar H^1 analogue of the paper's sesquilinear forms a, b, c of
Section 2, with the QEP written K + lambda C + lambda^2 M, Eq. (QuadEig)):

  K_ab = int grad B_a . grad B_b,   M_ab = int B_a B_b,
  C    = sum_e sigma_e M_e           (per-element damping coefficient).

Quadrature: nq Gauss--Legendre points per direction on every element; nq = p+1
integrates the polynomial integrands of M_e and K_e exactly on the uniform
affine elements used here.  The element loop is literal: for every element the
2-D sums over the nq x nq points are formed, then scattered into a sparse
matrix (scipy's COO -> CSR conversion adds duplicates).
"""
import numpy as np
import scipy.sparse as sp

from .bspline import Space1D


class Assembled:
    """CSR pattern shared by K, M, C plus their FP64 values."""

    def __init__(self, n, indptr, indices, K, M, C, space):
        self.n1 = n                # DOFs per direction
        self.N = n * n
        self.indptr = indptr
        self.indices = indices
        self.K, self.M, self.C = K, M, C   # scipy CSR, identical patterns
        self.space = space

    def Q(self, sigma):
        """Q(sigma) = sigma^2 M + sigma C + K (the benchmark spec's shifted matrix;
        Eq. (QuadEig) evaluated at the shift)."""
        return (sigma * sigma) * self.M + sigma * self.C + self.K


def assemble(ne, p, block, sigma_e, nq=None):
    """Assemble K, M and C for an ne x ne mesh of degree-p B-splines.

    block = 0 gives maximum-continuity IGA; block = b > 0 gives rIGA with C^0
    lines every b elements.  sigma_e has ne*ne entries, element ex + ne*ey.
    """
    nq = p + 1 if nq is None else nq
    sigma_e = np.asarray(sigma_e, dtype=np.float64).reshape(ne, ne)  # [ey, ex]
    sp1 = Space1D(ne, p, block)
    n, nf = sp1.n, sp1.n_full
    tabs = sp1.element_tables(nq)
    # Per-element 1-D tables stacked over elements: (ne, nq, p+1)
    IX = np.stack([t[0] for t in tabs])
    V = np.stack([t[1] for t in tabs])
    D = np.stack([t[2] for t in tabs])
    W = np.stack([t[3] for t in tabs])
    if IX.shape[1] != p + 1:
        raise AssertionError("each element must carry p+1 functions per direction")

    rows, cols, vk, vm, vc = [], [], [], [], []
    npl = p + 1
    for ey in range(ne):
        # B_a(x_q, y_r) with a = (ax, ay); all elements of this row at once.
        vy, dy, wy = V[ey], D[ey], W[ey]
        # values of the 2-D functions and their gradients at the points:
        # shape (ex, q, r, ax, ay)
        B = np.einsum('xqa,rb->xqrab', V, vy)
        Bx = np.einsum('xqa,rb->xqrab', D, vy)
        By = np.einsum('xqa,rb->xqrab', V, dy)
        w2 = np.einsum('xq,r->xqr', W, wy)
        Me = np.einsum('xqr,xqrab,xqrcd->xabcd', w2, B, B, optimize=True)
        Ke = (np.einsum('xqr,xqrab,xqrcd->xabcd', w2, Bx, Bx, optimize=True)
              + np.einsum('xqr,xqrab,xqrcd->xabcd', w2, By, By, optimize=True))
        Ce = sigma_e[ey][:, None, None, None, None] * Me
        # global full-function indices of the local functions
        gx = IX                               # (ex, ax)
        gy = IX[ey]                           # (ay,)
        gi = gx[:, :, None] + nf * gy[None, None, :]       # (ex, ax, ay)
        fi = np.broadcast_to(gi[:, :, :, None, None], (ne, npl, npl, npl, npl))
        fj = np.broadcast_to(gi[:, None, None, :, :], (ne, npl, npl, npl, npl))
        rows.append(fi.ravel())
        cols.append(fj.ravel())
        vk.append(Ke.ravel())
        vm.append(Me.ravel())
        vc.append(Ce.ravel())
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)

    # Dirichlet: drop every entry touching a boundary function, renumber.
    ri, rj = rows % nf, rows // nf
    ci, cj = cols % nf, cols // nf
    keep = ((ri > 0) & (ri < nf - 1) & (rj > 0) & (rj < nf - 1)
            & (ci > 0) & (ci < nf - 1) & (cj > 0) & (cj < nf - 1))
    r = (ri[keep] - 1) + n * (rj[keep] - 1)
    c = (ci[keep] - 1) + n * (cj[keep] - 1)
    N = n * n

    def to_csr(v):
        A = sp.coo_matrix((np.concatenate(v)[keep], (r, c)), shape=(N, N)).tocsr()
        A.sum_duplicates()
        A.sort_indices()
        return A

    K, M, C = to_csr(vk), to_csr(vm), to_csr(vc)
    for A in (M, C):
        if not (np.array_equal(A.indptr, K.indptr) and np.array_equal(A.indices, K.indices)):
            raise AssertionError("K, M and C must share one pattern")
    return Assembled(n, K.indptr.copy(), K.indices.copy(), K, M, C, sp1)
