"""Pins of the FP64 CPU oracle against facts it does not compute itself.

Each test ties one oracle function to something fixed outside it: numbers
the paper prints (tests/golden), a library routine that is an independent
definition (scipy's B-splines, LAPACK's dense QZ / symmetric eigensolver),
a closed form, an invariant or brute force on a tiny case.
"""
import os

import numpy as np
import pytest
import scipy.interpolate as si
import scipy.linalg as sla

from oracle import bspline, pattern
from oracle.assemble import assemble
from oracle.nd import symbolic, nd_boxes
from oracle.multifrontal import factorize, PivotError
from oracle import qep
from oracle.adjoint import damping_gradient, element_quadratic_forms
from oracle import gep
from paper_2112_14064_gb300 import workloads
from eigmatch import multiset_max_rel

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------- B-splines
@pytest.mark.parametrize("ne,p,block", [(8, 2, 4), (8, 3, 4), (12, 4, 4), (6, 3, 0)])
def test_basis_matches_scipy_bspline(ne, p, block):
    """Cox--de Boor values and derivatives == scipy's independent B-splines."""
    kn = bspline.knot_vector(ne, p, block)
    t = np.array([float(k) for k in kn])
    xs = np.random.default_rng(0).uniform(0, 1, 25)
    nf = bspline.n_functions(kn, p)
    spl = si.BSpline(t, np.eye(nf), p, extrapolate=False)
    dspl = spl.derivative()
    for x in xs:
        v, d = bspline.basis_and_derivative(kn, p, x)
        np.testing.assert_allclose(v, spl(x), rtol=0, atol=1e-13)
        np.testing.assert_allclose(d, dspl(x), rtol=1e-12, atol=1e-10)
        assert v.sum() == pytest.approx(1.0, abs=1e-14)   # partition of unity


def test_fig4_pattern_counts():
    """Knot multiplicities + support coupling reproduce Fig. 4's printed N, nnz."""
    for space, ne, p, block, N, nnz in _golden("fig4_pattern.txt"):
        assert pattern.hcurl_counts(int(ne), int(p), int(block)) == (int(N), int(nnz)), space


def test_riga_dof_counts_closed_form():
    """n = ne + p - 2 + (nb - 1)(p - 1) DOFs per direction after Dirichlet."""
    for ne, p, b in [(16, 2, 4), (256, 3, 16), (64, 3, 16), (512, 4, 32), (32, 5, 8)]:
        s = bspline.Space1D(ne, p, b)
        assert s.n == ne + p - 2 + (ne // b - 1) * (p - 1)
        assert len(s.c0_dofs) == ne // b - 1
    assert bspline.Space1D(256, 3, 0).n == 257


def test_maxwell_printed_value():
    """The analytic formula pi^2 (i^2 + j^2) gives the printed 10442.04."""
    (i, j, val, dec), = _golden("maxwell_mode.txt")
    assert round(np.pi ** 2 * (int(i) ** 2 + int(j) ** 2), int(dec)) == float(val)


# ---------------------------------------------------------------- assembly
def _scipy_1d(ne, p, block):
    """1-D mass and stiffness matrices from scipy B-splines and a Gauss rule
    with 2p+2 points per element (both exact for these piecewise
    polynomials), Dirichlet functions dropped."""
    kn = bspline.knot_vector(ne, p, block)
    t = np.array([float(k) for k in kn])
    nf = len(t) - p - 1
    g, w = np.polynomial.legendre.leggauss(2 * p + 2)
    xs = np.concatenate([(e + (g + 1) / 2) / ne for e in range(ne)])
    ws = np.concatenate([w / (2 * ne)] * ne)
    spl = si.BSpline(t, np.eye(nf), p, extrapolate=False)
    B = spl(xs).T
    D = spl.derivative()(xs).T
    M1 = (B * ws) @ B.T
    K1 = (D * ws) @ D.T
    return M1[1:-1, 1:-1], K1[1:-1, 1:-1]


@pytest.mark.parametrize("ne,p,block", [(8, 2, 4), (8, 3, 4), (8, 3, 0), (10, 4, 5)])
def test_assembly_tensor_structure(ne, p, block):
    """With constant damping c: M = M1 (x) M1, K = M1 (x) K1 + K1 (x) M1,
    C = c M, where M1, K1 come from scipy's B-splines (DOF i + n j)."""
    c = 0.7
    A = assemble(ne, p, block, np.full(ne * ne, c))
    M1, K1 = _scipy_1d(ne, p, block)
    np.testing.assert_allclose(A.M.toarray(), np.kron(M1, M1), rtol=0, atol=1e-15)
    np.testing.assert_allclose(A.K.toarray(), np.kron(M1, K1) + np.kron(K1, M1),
                               rtol=0, atol=1e-12)
    np.testing.assert_allclose(A.C.toarray(), c * A.M.toarray(), rtol=1e-14, atol=1e-17)
    nnz = pattern.h1_counts(ne, p, block)[1]
    assert A.K.nnz == nnz


def test_damping_single_element():
    """sigma_e = indicator of one element: C is that element's mass matrix,
    the product of the 1-D element mass matrices."""
    ne, p, b = 8, 3, 4
    e0x, e0y = 3, 5
    s = np.zeros(ne * ne)
    s[e0x + ne * e0y] = 1.0
    A = assemble(ne, p, b, s)
    kn = bspline.knot_vector(ne, p, b)
    t = np.array([float(k) for k in kn])
    nf = len(t) - p - 1
    g, w = np.polynomial.legendre.leggauss(2 * p + 2)

    spl = si.BSpline(t, np.eye(nf), p, extrapolate=False)

    def m1(e):
        xs = (e + (g + 1) / 2) / ne
        B = spl(xs).T
        return ((B * (w / (2 * ne))) @ B.T)[1:-1, 1:-1]

    np.testing.assert_allclose(A.C.toarray(), np.kron(m1(e0y), m1(e0x)), atol=1e-16)


def test_undamped_limit_converges_to_laplacian():
    """sigma_e = 0: -lambda^2 = mu_h -> pi^2 (m^2 + n^2) at order ~2p."""
    p = 2
    exact = np.pi ** 2 * np.array(sorted(m * m + n * n for m in range(1, 5)
                                         for n in range(1, 5)))[:6]
    errs = []
    for ne in (8, 16):
        A = assemble(ne, p, 4, np.zeros(ne * ne))
        mu = sla.eigh(A.K.toarray(), A.M.toarray(), eigvals_only=True)[:6]
        errs.append(np.abs(mu - exact) / exact)
    order = np.log2(errs[0] / errs[1])
    assert np.all(errs[1] < 1e-3)
    assert np.all(order > 2 * p - 0.6), order


# ---------------------------------------------------------------- symbolic
def _brute_symbolic(A, sym):
    """Column structures of L by dense boolean elimination."""
    N = A.N
    P = (A.K.toarray() != 0)[np.ix_(sym.perm, sym.perm)]
    S = P.copy()
    for j in range(N):
        rows = np.flatnonzero(S[j + 1:, j]) + j + 1
        S[np.ix_(rows, rows)] = True
    return S


@pytest.mark.parametrize("ne,p,block", [(16, 2, 4), (8, 3, 4), (10, 2, 0)])
def test_symbolic_against_brute_force(ne, p, block):
    A = assemble(ne, p, block, np.ones(ne * ne))
    sym = symbolic(A.n1, A.space.c0_dofs, p, A.indptr, A.indices, use_c0=block > 0)
    N = A.N
    assert sorted(sym.perm.tolist()) == list(range(N))
    S = _brute_symbolic(A, sym)
    for s in range(sym.nsuper):
        a, e = sym.sptr[s], sym.sptr[s + 1]
        exact = np.flatnonzero(S[e:, a:e].any(axis=1)) + e
        np.testing.assert_array_equal(sym.struct(s), exact)
        if sym.parent[s] >= 0:
            assert sym.parent[s] > s
            pa = sym.parent[s]
            assert sym.sptr[pa] <= sym.struct(s)[0] < sym.sptr[pa + 1]
        # every struct entry belongs to an ancestor's pivots
        anc = set()
        q = sym.parent[s]
        while q >= 0:
            anc |= set(range(sym.sptr[q], sym.sptr[q + 1]))
            q = sym.parent[q]
        assert set(sym.struct(s).tolist()) <= anc


def test_separators_separate():
    """No matrix entry couples the two children of a dissection cut."""
    ne, p, b = 16, 3, 8
    A = assemble(ne, p, b, np.ones(ne * ne))
    n = A.n1
    boxes = nd_boxes(n, A.space.c0_dofs, p)
    Kd = A.K.toarray() != 0
    # within a macroelement the p-wide cut separates; the C^0 line too
    for (x0, x1, y0, y1) in boxes:
        if x1 - x0 in (1, p) and y1 - y0 > p:
            lo = [xx + n * yy for yy in range(y0, y1) for xx in range(max(0, x0 - 3 * p), x0)]
            hi = [xx + n * yy for yy in range(y0, y1) for xx in range(x1, min(n, x1 + 3 * p))]
            if lo and hi:
                assert not Kd[np.ix_(lo, hi)].any()


def test_nd_cut_rule_hand_derived_riga_ties():
    """Canonical cut rule against a box list worked out by hand.

    ne = 12, p = 2, blocks of 4: n = 14 DOFs per direction and the C^0
    functions of the knots 4/12 and 8/12 are DOFs 4 and 9 (a block of b
    elements with C^0 ends holds b + p - 2 interior functions, so the k-th
    C^0 function is full index k (b + p - 1), DOF index one less).  The
    centre of [0, 14) is 6.5, equidistant from 4 and 9: every tie goes to
    the lower line.  Root: both directions C^0-cuttable, equal extents, so
    x is cut at 4.  Low child [0,4)x[0,14): only y has lines inside (4 and
    9, tie -> 4), then [0,4)x[5,14) is cut at 9.  High child [5,14)x[0,14):
    x has 9 inside, y has 4 and 9; y is longer, cut at 4 (tie); then
    [5,14)x[0,4) is cut in x at 9, [5,14)x[5,14) in x at 9 (equal extents),
    and each half of it in y at 9.  Boxes of extent <= 8 without a C^0 line
    inside are leaves."""
    got = nd_boxes(14, [4, 9], 2)
    want = [(0, 4, 0, 4), (0, 4, 5, 9), (0, 4, 10, 14), (0, 4, 9, 10), (0, 4, 4, 5),
            (5, 9, 0, 4), (10, 14, 0, 4), (9, 10, 0, 4),
            (5, 9, 5, 9), (5, 9, 10, 14), (5, 9, 9, 10),
            (10, 14, 5, 9), (10, 14, 10, 14), (10, 14, 9, 10), (9, 10, 5, 14),
            (5, 14, 4, 5), (4, 5, 0, 14)]
    assert got == want
    # the C^0 DOF indices above are those of the oracle's knot logic
    assert bspline.Space1D(12, 2, 4).c0_dofs == [4, 9]


@pytest.mark.parametrize("n,want", [
    # extent 10 > 8: p-wide cut at 0 + (10 - 2) // 2 = 4 (tie of extents -> x),
    # then each 4 x 10 half is cut in y at 4, leaving 4 x 4 leaves
    (10, [(0, 4, 0, 4), (0, 4, 6, 10), (0, 4, 4, 6), (6, 10, 0, 4), (6, 10, 6, 10),
          (6, 10, 4, 6), (4, 6, 0, 10)]),
    # extent 11: the cut starts at (11 - 2) // 2 = 4 (floor), the high half
    # keeps the odd extent 5
    (11, [(0, 4, 0, 4), (0, 4, 6, 11), (0, 4, 4, 6), (6, 11, 0, 4), (6, 11, 6, 11),
          (6, 11, 4, 6), (4, 6, 0, 11)]),
])
def test_nd_cut_rule_hand_derived_iga(n, want):
    """IGA (no C^0 lines): only the p-wide cuts of the macroelement rule."""
    assert nd_boxes(n, [], 2) == want


def _brute_counts(A, sym):
    """Exact column counts and the supernodal counts from dense boolean
    elimination of the stored pattern (numerically zero entries of K, where
    gradients cancel, are still stored entries): c_j = structurally non-zero rows below j in column j; a
    supernode stores its dense lower pivot triangle and every row below the
    block that is non-zero in any of its columns."""
    N = A.N
    P = np.zeros((N, N), dtype=bool)               # the stored (CSR) pattern
    for i in range(N):
        P[i, A.indices[A.indptr[i]:A.indptr[i + 1]]] = True
    S = P[np.ix_(sym.perm, sym.perm)]
    for j in range(N):
        rows = np.flatnonzero(S[j + 1:, j]) + j + 1
        S[np.ix_(rows, rows)] = True
    c = np.array([int(S[j + 1:, j].sum()) for j in range(N)])
    nnz_sup, fl_sup = 0, 0
    for s in range(sym.nsuper):
        a, e = int(sym.sptr[s]), int(sym.sptr[s + 1])
        k = e - a
        u = int(S[e:, a:e].any(axis=1).sum())
        nnz_sup += k * (k + 1) // 2 + k * u
        fl_sup += sum((k - 1 - t + u) ** 2 + 2 * (k - 1 - t + u) for t in range(k))
    return c, nnz_sup, fl_sup


@pytest.mark.parametrize("ne,p,block", [(16, 2, 4), (8, 2, 4), (8, 3, 4), (10, 2, 0)])
def test_factor_counts_against_brute_force(ne, p, block):
    """nnz(L) and the Cholesky flop count sum_j (c_j^2 + 2 c_j), both in their
    exact (scalar) form and in the supernodal form with dense pivot blocks,
    equal the counts of a dense boolean elimination of the ordered pattern."""
    A = assemble(ne, p, block, np.ones(ne * ne))
    sym = symbolic(A.n1, A.space.c0_dofs, p, A.indptr, A.indices, use_c0=block > 0)
    c, nnz_sup, fl_sup = _brute_counts(A, sym)
    np.testing.assert_array_equal(sym.scalar_col_counts(A.indptr, A.indices), c)
    assert sym.nnz_L_scalar(A.indptr, A.indices) == int((c + 1).sum())
    assert sym.factor_flops_scalar(A.indptr, A.indices) == int((c * c + 2 * c).sum())
    assert sym.nnz_L() == nnz_sup
    assert sym.factor_flops() == fl_sup
    # dense pivot blocks hold explicit zeros: the supernodal count is larger
    assert sym.nnz_L() >= sym.nnz_L_scalar(A.indptr, A.indices)


# ---------------------------------------------------------------- factor
@pytest.mark.parametrize("ne,p,block", [(16, 2, 4), (8, 3, 4), (8, 3, 0)])
def test_ldlt_reconstructs_Q(ne, p, block):
    sig = workloads.sigma_e(dict(ne=ne, sigma_law="uniform", lo=0.1, hi=1.0, seed=1))
    A = assemble(ne, p, block, sig)
    sym = symbolic(A.n1, A.space.c0_dofs, p, A.indptr, A.indices, use_c0=block > 0)
    Q = A.Q(20.0)
    F = factorize(sym, Q)
    N = A.N
    L = np.zeros((N, N))
    for s in range(sym.nsuper):
        a, e = sym.sptr[s], sym.sptr[s + 1]
        idx = np.concatenate([np.arange(a, e), sym.struct(s)])
        L[np.ix_(idx, np.arange(a, e))] = F.L[s]
    Qp = Q.toarray()[np.ix_(sym.perm, sym.perm)]
    R = L @ np.diag(F.D) @ L.T - Qp
    assert np.abs(R).max() / np.abs(Qp).max() < 1e-14
    b = np.random.default_rng(2).standard_normal(N)
    x = F.solve(b)
    np.testing.assert_allclose(x, np.linalg.solve(Q.toarray(), b), rtol=1e-11, atol=0)


def test_non_positive_pivot_is_reported():
    """A shifted matrix that is not positive definite stops the oracle."""
    A = assemble(8, 2, 4, np.ones(64))
    sym = symbolic(A.n1, A.space.c0_dofs, 2, A.indptr, A.indices)
    with pytest.raises(PivotError):
        factorize(sym, -1.0 * A.K)


# ---------------------------------------------------------------- operator
def test_block_operator_solves_linearised_pencil():
    """Eq. (BlockOperatorVector): L(s) r = B v with the dense 2N pencil."""
    ne, p, b, s = 16, 2, 4, 20.0
    cfg = workloads.CONFIGS["tiny"]
    A = assemble(ne, p, b, workloads.sigma_e(cfg))
    sym = symbolic(A.n1, A.space.c0_dofs, p, A.indptr, A.indices)
    F = factorize(sym, A.Q(s))
    N = A.N
    v = workloads.start_vector(3, 2 * N)
    r = qep.apply_operator(v, s, A.M, A.C, F.solve)
    K, C, M = A.K.toarray(), A.C.toarray(), A.M.toarray()
    I, Z = np.eye(N), np.zeros((N, N))
    Amat = np.block([[Z, I], [-K, -C]])
    Bmat = np.block([[I, Z], [Z, M]])
    Ls = Amat - s * Bmat
    res = Ls @ r - Bmat @ v
    assert np.linalg.norm(res) / np.linalg.norm(Bmat @ v) < 1e-13


# ---------------------------------------------------------------- eigs
def _dense_nearest(A, s, neig):
    N = A.N
    K, C, M = A.K.toarray(), A.C.toarray(), A.M.toarray()
    I, Z = np.eye(N), np.zeros((N, N))
    w = sla.eig(np.block([[Z, I], [-K, -C]]), np.block([[I, Z], [Z, M]]), right=False)
    return w[qep.wanted_order(w, s)][:neig]


def _solve_tiny(cfg_over=None, s=None, neig=None, m=None):
    cfg = dict(workloads.CONFIGS["tiny"])
    if cfg_over:
        cfg.update(cfg_over)
    A = assemble(cfg["ne"], cfg["p"], cfg["block"], workloads.sigma_e(cfg))
    sym = symbolic(A.n1, A.space.c0_dofs, cfg["p"], A.indptr, A.indices)
    s = cfg["shift"] if s is None else s
    F = factorize(sym, A.Q(s))
    r = qep.eigs(A.K, A.C, A.M, s, neig or cfg["neig"], m or cfg["m"], F.solve,
                 workloads.start_vector(1, 2 * A.N))
    return A, r


def test_eigs_match_dense_qz():
    """P-1: nearest eigenvalues of the 2N pencil by LAPACK's QZ."""
    A, r = _solve_tiny()
    assert r.n_conv == 10
    ref = _dense_nearest(A, 20.0, 10)
    assert multiset_max_rel(ref, r.lam) < 1e-10
    # locked pairs stop at the convergence tolerance; the target is eta <= 1e-10
    assert np.all(r.eta <= 1e-10)


def test_proportional_damping_closed_form():
    """P-2: C = cM gives lambda = (-c +- sqrt(c^2 - 4 mu)) / 2 for each mu of
    K x = mu M x (LAPACK's symmetric-definite solver)."""
    c = 0.4
    A, r = _solve_tiny({"sigma_law": "constant", "value": c})
    mu = sla.eigh(A.K.toarray(), A.M.toarray(), eigvals_only=True)
    disc = np.sqrt((c * c - 4 * mu).astype(complex))
    lam_all = np.concatenate([(-c + disc) / 2, (-c - disc) / 2])
    assert r.n_conv == 10
    assert multiset_max_rel(lam_all, r.lam) < 1e-10


def test_undamped_eigs_are_imaginary():
    """sigma_e = 0: lambda = +- i sqrt(mu_h)."""
    A, r = _solve_tiny({"sigma_law": "constant", "value": 0.0})
    mu = sla.eigh(A.K.toarray(), A.M.toarray(), eigvals_only=True)
    lam_all = np.concatenate([1j * np.sqrt(mu), -1j * np.sqrt(mu)])
    assert multiset_max_rel(lam_all, r.lam) < 1e-10
    assert np.max(np.abs(r.lam.real)) < 1e-8


def test_backward_error_detects_wrong_eigenvalue():
    A, r = _solve_tiny()
    lam, x = r.lam[0], r.X[0]
    assert qep.backward_error(lam, x, A.K, A.C, A.M) < 1e-12
    assert qep.backward_error(lam * (1 + 1e-6), x, A.K, A.C, A.M) > 1e-9


def test_eigenvector_normalisation():
    A, r = _solve_tiny()
    for x in r.X:
        assert np.linalg.norm(x) == pytest.approx(1.0, abs=1e-14)
        i = np.argmax(np.abs(x))
        assert abs(x[i].imag) < 1e-15 and x[i].real > 0


def _dense_all(A):
    """Every eigenvalue of the 2N pencil (A, B) = ([[0, I], [-K, -C]],
    diag(I, M)).  B is invertible, so they are the eigenvalues of
    B^{-1}A = [[0, I], [-M^{-1}K, -M^{-1}C]] (LAPACK's dgeev; M^{-1} applied
    by a Cholesky solve), about 50 times faster than QZ at 2N = 2450."""
    N = A.N
    K, C, M = A.K.toarray(), A.C.toarray(), A.M.toarray()
    cf = sla.cho_factor(M)
    I, Z = np.eye(N), np.zeros((N, N))
    return np.linalg.eigvals(np.block([[Z, I], [-sla.cho_solve(cf, K), -sla.cho_solve(cf, C)]]))


_INREGION = {}


def _inregion_problem(ne, p, block, seed):
    key = (ne, p, block, seed)
    if key not in _INREGION:
        cfg = dict(ne=ne, p=p, block=block, sigma_law="uniform", lo=0.1, hi=1.0, seed=seed)
        sig = workloads.sigma_e(cfg)
        A = assemble(ne, p, block, sig)
        sym = symbolic(A.n1, A.space.c0_dofs, p, A.indptr, A.indices)
        F = factorize(sym, A.Q(0.0))
        _INREGION[key] = (A, sig, F, _dense_all(A))
    return _INREGION[key]


@pytest.mark.parametrize("mesh,neig,target,ncand,m,certified", [
    ((16, 2, 4, 20211228), 10, 20.0, 16, 40, True),
    ((16, 2, 4, 20211228), 10, 20.0, 10, 30, False),    # too few candidates
    ((16, 2, 4, 20211228), 10, 300.0, 40, 80, True),
    ((32, 3, 16, 20211232), 20, 500.0, 80, 120, True),
    ((32, 3, 16, 20211232), 20, 800.0, 80, 120, True),
    ((32, 3, 16, 20211232), 20, 2000.0, 20, 40, False),  # too few candidates
])
def test_in_region_selection_against_dense(mesh, neig, target, ncand, m, certified):
    """Shift inside the spectrum region (shift 0, Section 4.1.4), neig pairs
    nearest a real target chosen among ncand converged candidates, against
    every eigenvalue of the dense pencil.

    * The facts the certificate rests on hold for the dense spectrum:
      complex eigenvalues have Re in [-max sigma_e / 2, -min sigma_e / 2],
      real ones are <= 0, and every eigenvalue within r (the largest
      candidate distance from the shift) is a candidate.
    * A certified selection is the multiset of the neig eigenvalues nearest
      the target (1e-10 relative).
    * The uncertified cases return a wrong selection: the certificate is not
      vacuous there (a sign slip making it more permissive would certify
      them and fail)."""
    A, sig, F, w = _inregion_problem(*mesh)
    cplx = np.abs(w.imag) > 0
    assert np.all(w[cplx].real <= -sig.min() / 2 * (1 - 1e-9))
    assert np.all(w[cplx].real >= -sig.max() / 2 * (1 + 1e-9))
    assert np.all(w[~cplx].real <= 1e-9)
    r = qep.eigs(A.K, A.C, A.M, 0.0, neig, m, F.solve, workloads.start_vector(1, 2 * A.N),
                 target=target, ncand=ncand, sigma_min=sig.min())
    assert r.certified == certified
    rad = np.abs(r.candidates).max()
    inside = w[np.abs(w) < rad * (1 - 1e-9)]
    assert multiset_max_rel(r.candidates, inside) < 1e-9      # Krylov found them all
    ref = w[qep.wanted_order(w, target)][:neig]
    err = multiset_max_rel(ref, r.lam)
    if certified:
        assert err < 1e-10
        assert np.all(r.eta <= 1e-10)
    else:
        assert err > 1e-6


def test_scaled_pencil_same_eigenvalues():
    """Remark 4's scaling is an exact change of variable: the scaled oracle
    returns the dense pencil's eigenvalues (literal shift 20 and the
    in-region shift with target 300), and varsigma is the square root of the
    ratio of the largest entries of K and M."""
    A, _ = _solve_tiny()
    vs = qep.scaling_factor(A.K, A.M)
    assert vs == pytest.approx(np.sqrt(np.abs(A.K.toarray()).max() / np.abs(A.M.toarray()).max()))
    assert vs > 10.0      # K and M differ by orders of magnitude here
    sym = symbolic(A.n1, A.space.c0_dofs, 2, A.indptr, A.indices)
    v1 = workloads.start_vector(1, 2 * A.N)
    F = factorize(sym, A.Q(20.0))
    r = qep.eigs_scaled(A.K, A.C, A.M, 20.0, 10, 40, F.solve, v1)
    assert multiset_max_rel(_dense_nearest(A, 20.0, 10), r.lam) < 1e-10
    assert np.all(r.eta <= 1e-10)
    sig = workloads.sigma_e(workloads.CONFIGS["tiny"])
    F0 = factorize(sym, A.Q(0.0))
    r = qep.eigs_scaled(A.K, A.C, A.M, 0.0, 10, 80, F0.solve, v1, target=300.0, ncand=40,
                        sigma_min=sig.min())
    assert r.certified
    assert multiset_max_rel(_dense_nearest(A, 300.0, 10), r.lam) < 1e-10


@pytest.mark.parametrize("ne,p,block", [(16, 2, 4), (12, 3, 0)])
def test_inertia_counts_eigenvalues_below(ne, p, block):
    """Sylvester's law (Section 4.1.4): the negative pivots of the no-pivot
    LDL^T of K - mu M count the eigenvalues of K x = mu' M x below mu,
    compared with LAPACK's symmetric-definite solver."""
    A = assemble(ne, p, block, np.zeros(ne * ne))
    sym = symbolic(A.n1, A.space.c0_dofs, p, A.indptr, A.indices, use_c0=block > 0)
    mu_all = sla.eigh(A.K.toarray(), A.M.toarray(), eigvals_only=True)
    for mu in (1.0, 30.0, 123.4, 700.0, 5000.0):
        assert gep.inertia(sym, A.K, A.M, mu) == int((mu_all < mu).sum()), mu


def test_lanczos_slice_against_dense():
    """Spectrum slicing: the eigenvalues in [100, 400) (with the x <-> y
    double eigenvalues of the square) by inertia counts and shift-and-invert
    Lanczos at the midpoint, against LAPACK; the slice is certified and every
    pair has a residual below 1e-10.  When Lanczos is asked for one pair
    fewer than the inertia count, the count check fails and the slice is
    not certified (a missed eigenvalue is caught)."""
    A = assemble(16, 2, 4, np.zeros(256))
    sym = symbolic(A.n1, A.space.c0_dofs, 2, A.indptr, A.indices)
    mu_all = sla.eigh(A.K.toarray(), A.M.toarray(), eigvals_only=True)
    v1 = workloads.start_vector(1, A.N)
    mus, X, count, cert = gep.slice(sym, A.K, A.M, 100.0, 400.0, 40, v1)
    ref = mu_all[(mu_all >= 100.0) & (mu_all < 400.0)]
    assert cert and count == len(ref) == len(mus)
    assert multiset_max_rel(ref, mus) < 1e-10
    assert max(gep.residual(A.K, A.M, m_, x) for m_, x in zip(mus, X)) <= 1e-10
    mus, X, count, cert = gep.slice(sym, A.K, A.M, 100.0, 400.0, 40, v1, extra=-1)
    assert count == len(ref) and len(mus) == count - 1
    assert not cert


@pytest.mark.parametrize("shift", [1j * np.sqrt(300.0), 0.2 + 1j * np.sqrt(120.0)])
def test_complex_shift_against_dense(shift):
    """Section 4.1.1's complex shift: the complex symmetric LDL^T solves
    Q(s) x = b, and the real-operator Krylov-Schur with the quadratic
    back-mapping returns the eigenvalues of the dense pencil nearest s
    (LAPACK's QZ, multiset 1e-10)."""
    c = workloads.CONFIGS["tiny"]
    A = assemble(c["ne"], c["p"], c["block"], workloads.sigma_e(c))
    sym = symbolic(A.n1, A.space.c0_dofs, c["p"], A.indptr, A.indices)
    Q = (A.K + shift * A.C + shift * shift * A.M).tocsr()
    F = factorize(sym, Q)
    rng = np.random.default_rng(1)
    b = rng.standard_normal(A.N) + 1j * rng.standard_normal(A.N)
    assert np.linalg.norm(Q @ F.solve(b) - b) <= 1e-13 * np.linalg.norm(b)
    r = qep.eigs_complex_shift(A.K, A.C, A.M, shift, 10, 40, F.solve,
                               workloads.start_vector(1, 2 * A.N))
    N = A.N
    K, C, M = A.K.toarray(), A.C.toarray(), A.M.toarray()
    I, Z = np.eye(N), np.zeros((N, N))
    w = sla.eig(np.block([[Z, I], [-K, -C]]), np.block([[I, Z], [Z, M]]), right=False)
    ref = w[np.lexsort((-w.imag, np.abs(w - shift)))][:10]
    assert multiset_max_rel(ref, r.lam) < 1e-10
    assert np.all(r.eta <= 1e-10)


# ---------------------------------------------------------------- gradient
def test_gradient_sum_rule_proportional():
    """P-2: with C = cM, sum_e dlambda/dsigma_e = -lambda / (2 lambda + c),
    from differentiating lambda^2 + c lambda + mu = 0 in c."""
    c = 0.4
    A, r = _solve_tiny({"sigma_law": "constant", "value": c})
    cfg = workloads.CONFIGS["tiny"]
    G = damping_gradient(cfg["ne"], cfg["p"], cfg["block"], r.lam[:4], r.X[:4], A.C, A.M)
    for lam, g in zip(r.lam[:4], G):
        assert g.sum() == pytest.approx(-lam / (2 * lam + c), rel=1e-9)


def test_element_forms_sum_to_mass_form():
    """sum_e x_e^T M_e x_e = x^T M x (the element forms partition M)."""
    cfg = workloads.CONFIGS["tiny"]
    A = assemble(cfg["ne"], cfg["p"], cfg["block"], np.ones(cfg["ne"] ** 2))
    x = np.random.default_rng(4).standard_normal(A.N) + 1j * np.random.default_rng(5).standard_normal(A.N)
    q = element_quadratic_forms(cfg["ne"], cfg["p"], cfg["block"], x)
    assert q.sum() == pytest.approx(x @ (A.M @ x), rel=1e-13)


def test_gradient_central_differences():
    """P-8: analytic dlambda/dsigma_e vs central differences of the dense-QZ
    eigenvalue tracked by nearest match.  The step is 1e-4: the gradients are
    ~1e-5 while QZ's eigenvalues carry ~1e-13 absolute rounding, so a 1e-6
    step would leave ~1e-3 relative noise; at 1e-4 the O(h^2) truncation
    and the rounding are both below 1e-6 relative."""
    ne, p, b, s = 8, 2, 4, 20.0
    cfg = dict(ne=ne, sigma_law="uniform", lo=0.1, hi=1.0, seed=11)
    sig = workloads.sigma_e(cfg)
    A = assemble(ne, p, b, sig)
    sym = symbolic(A.n1, A.space.c0_dofs, p, A.indptr, A.indices)
    F = factorize(sym, A.Q(s))
    r = qep.eigs(A.K, A.C, A.M, s, 4, 20, F.solve, workloads.start_vector(1, 2 * A.N))
    G = damping_gradient(ne, p, b, r.lam, r.X, A.C, A.M)
    h = 1e-4
    for e in (0, 9, 27, 63):
        fd = []
        for sgn in (+1, -1):
            s2 = sig.copy()
            s2[e] += sgn * h
            A2 = assemble(ne, p, b, s2)
            w = _dense_nearest(A2, s, 8)
            fd.append([w[np.argmin(np.abs(w - l))] for l in r.lam])
        fd = (np.array(fd[0]) - np.array(fd[1])) / (2 * h)
        # atol: ~1e-13 QZ rounding / (2h) = 5e-10, with a factor 4 margin
        np.testing.assert_allclose(G[:, e], fd, rtol=1e-5, atol=2e-9)
