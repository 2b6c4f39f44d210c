"""Univariate B-spline spaces for IGA and rIGA (oracle; test infrastructure only).

Plain, slow FP64 restatement of Section 3 of the paper:

* open knot vectors, Eqs. (KnotsX)/(KnotsY), Section 3.1;
* Cox--de Boor recursion, Eqs. (BasisFunBi0)/(BasisFunBip), with the
  convention that a 0/0 quotient is 0 (the paper's "avoiding any division by
  zero", Section 3.1);
* rIGA: interior knots on macroelement boundaries repeated p times, which
  makes the space C^0 there (Section 3.3; scalar H^1 form of the refinement the
  paper cites for H^1 spaces);
* homogeneous Dirichlet condition: the first and last functions of an open
  knot vector are the only ones that do not vanish on the boundary, so they
  are dropped.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.
"""
from fractions import Fraction

import numpy as np


def knot_vector(ne, p, block=0, sep_mult=None):
    """Open knot vector on [0, 1] with ``ne`` uniform elements.

    Interior knot k/ne has multiplicity 1 (maximum continuity C^{p-1}, IGA,
    Section 3.2) unless ``block > 0`` and k is a multiple of ``block``: then
    its multiplicity is ``sep_mult`` (default p: continuity C^0 across the
    macroelement boundary, rIGA, Section 3.3).  Knots are exact rationals (Fraction) so that knot
    comparisons are exact; they are converted to float only for evaluation.
    """
    if p < 1 or ne < 1:
        raise ValueError("need p >= 1 and ne >= 1")
    if block and ne % block:
        raise ValueError("ne must be a multiple of the block size")
    sep_mult = p if sep_mult is None else sep_mult
    t = [Fraction(0)] * (p + 1)
    for k in range(1, ne):
        mult = sep_mult if (block and k % block == 0) else 1
        t += [Fraction(k, ne)] * mult
    t += [Fraction(1)] * (p + 1)
    return t


def n_functions(knots, p):
    """Number of B-splines of degree p on a knot vector: len(knots) - p - 1."""
    return len(knots) - p - 1


def _ratio(num, den):
    # Cox--de Boor with repeated knots: a term whose denominator vanishes is
    # multiplied by a zero-width lower-degree function and is taken as 0.
    return 0.0 if den == 0 else num / den


def basis_all(knots, p, x):
    """Values of every degree-p B-spline at x, straight from the recursion.

    Degree 0 (Eq. BasisFunBi0): N_i^0(x) = 1 on [t_i, t_{i+1}), else 0, with
    the last non-empty span closed on the right so that x = 1 is covered.
    Degree q (Eq. BasisFunBip):
      N_i^q = (x - t_i)/(t_{i+q} - t_i) N_i^{q-1}
            + (t_{i+q+1} - x)/(t_{i+q+1} - t_{i+1}) N_{i+1}^{q-1}.
    Returns (values of degree p, values of degree p-1) as float arrays.
    """
    t = [float(k) for k in knots]
    m = len(t) - 1
    last = max(i for i in range(m) if t[i] < t[i + 1])
    N = np.zeros(m)
    for i in range(m):
        if t[i] <= x < t[i + 1] or (i == last and x == t[i + 1]):
            N[i] = 1.0
    prev = N
    for q in range(1, p + 1):
        cur = np.zeros(m - q)
        for i in range(m - q):
            cur[i] = (_ratio(x - t[i], t[i + q] - t[i]) * prev[i]
                      + _ratio(t[i + q + 1] - x, t[i + q + 1] - t[i + 1]) * prev[i + 1])
        if q == p:
            return cur, prev[: m - q + 1]
        prev = cur
    return prev, None  # p == 0


def basis_and_derivative(knots, p, x):
    """Values and first derivatives of all degree-p B-splines at x.

    The derivative is the standard consequence of the recursion:
      dN_i^p/dx = p/(t_{i+p} - t_i) N_i^{p-1} - p/(t_{i+p+1} - t_{i+1}) N_{i+1}^{p-1}.
    """
    t = [float(k) for k in knots]
    vals, low = basis_all(knots, p, x)
    n = len(vals)
    der = np.zeros(n)
    for i in range(n):
        der[i] = (p * _ratio(1.0, t[i + p] - t[i]) * low[i]
                  - p * _ratio(1.0, t[i + p + 1] - t[i + 1]) * low[i + 1])
    return vals, der


def supports(knots, p):
    """Support [t_i, t_{i+p+1}] of each function, as exact rationals."""
    return [(knots[i], knots[i + p + 1]) for i in range(n_functions(knots, p))]


def coupled(knots, p, i, j):
    """True when functions i and j overlap on a set of positive length.

    Two B-splines couple in a Galerkin matrix exactly when their supports
    share an open interval; this is what decides the sparsity pattern.
    """
    a0, a1 = knots[i], knots[i + p + 1]
    b0, b1 = knots[j], knots[j + p + 1]
    return max(a0, b0) < min(a1, b1)


def c0_functions(knots, p):
    """Indices of the functions that sit on a C^0 interior knot.

    A function N_i whose interior knots t_{i+1} .. t_{i+p} are one repeated
    interior knot value is the only function that does not vanish there;
    in rIGA these form the one-DOF-thick separators (Section 3.3).
    """
    out = []
    for i in range(n_functions(knots, p)):
        inner = knots[i + 1: i + p + 1]
        if p >= 2 and len(set(inner)) == 1 and 0 < inner[0] < 1:
            out.append(i)
    return out


def gauss_legendre(nq):
    """Gauss--Legendre points and weights on [-1, 1] (numpy's leggauss)."""
    return np.polynomial.legendre.leggauss(nq)


class Space1D:
    """One direction of the tensor-product space, Dirichlet functions removed.

    DOF d of this direction is full function d + 1 (the first and last
    functions of the open knot vector are dropped).
    """

    def __init__(self, ne, p, block=0):
        self.ne, self.p, self.block = ne, p, block
        self.knots = knot_vector(ne, p, block)
        self.n_full = n_functions(self.knots, p)
        self.n = self.n_full - 2
        self.c0_dofs = [i - 1 for i in c0_functions(self.knots, p)
                        if 1 <= i <= self.n_full - 2]

    def dof_coupled(self, a, b):
        return coupled(self.knots, self.p, a + 1, b + 1)

    def element_tables(self, nq):
        """Per element: nonzero full-function indices and their values and
        derivatives at the nq mapped Gauss points, plus the mapped weights.

        Element ex covers [ex/ne, (ex+1)/ne]; the geometric map is the
        identity on the unit square so parametric derivatives are physical.
        """
        g, w = gauss_legendre(nq)
        h = 1.0 / self.ne
        tabs = []
        for ex in range(self.ne):
            xs = (ex + (g + 1.0) / 2.0) * h
            ws = w * h / 2.0
            vals = np.zeros((nq, self.n_full))
            ders = np.zeros((nq, self.n_full))
            for q, x in enumerate(xs):
                vals[q], ders[q] = basis_and_derivative(self.knots, self.p, x)
            nz = [i for i in range(self.n_full) if np.any(vals[:, i] != 0.0)
                  or np.any(ders[:, i] != 0.0)]
            tabs.append((np.array(nz), vals[:, nz], ders[:, nz], ws))
        return tabs
