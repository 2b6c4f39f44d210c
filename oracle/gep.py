"""Undamped problem: Lanczos and spectrum slicing (oracle).

Plain FP64 restatement, test infrastructure only.

Without damping the QEP (lambda^2 M + K) u = 0 is the symmetric-definite
generalized eigenproblem K x = mu M x with lambda = +-i sqrt(mu).  For such
pencils the paper reviews (Section 4.1.4) spectrum slicing: by Sylvester's
law of inertia, the number of eigenvalues mu < sigma equals the number of
negative entries of D in K - sigma M = L D L^T, so the eigenvalues in an
interval [a, b) are counted by two factorisations; and Lanczos (Remark 3):
with a Hermitian operator and a real shift the Arnoldi recurrence
orthogonalises only against the last two vectors and H is symmetric
tridiagonal.

* inertia(sym, K, M, mu): negative pivots of the LDL^T of K - mu M.
* lanczos(K, M, sigma, ...): shift-and-invert Lanczos on
  op = (K - sigma M)^{-1} M in the M-inner product (self-adjoint there),
  theta = 1/(mu - sigma).  The three-term recurrence of Remark 3 is run with
  full reorthogonalisation (classical Gram-Schmidt twice against every
  basis vector, which keeps the computed basis orthogonal; the coefficients
  outside the tridiagonal band are then rounding) and thick restarts (the
  symmetric counterpart of Krylov-Schur: the k Ritz vectors nearest sigma
  are kept).
* slice(...): eigenpairs with mu in [a, b), counted by inertia, computed by
  Lanczos at the interval's midpoint; certified when Lanczos returns exactly
  the counted number of eigenvalues in the interval.
"""
import numpy as np

from .multifrontal import factorize


def inertia(sym, K, M, mu):
    """Number of eigenvalues of K x = mu' M x with mu' < mu (Sylvester)."""
    F = factorize(sym, (K - mu * M).tocsr(), indefinite=True)
    return int((F.D < 0).sum())


def lanczos(K, M, sigma, nwant, m, solve, v1, tol=1e-10, max_restarts=500):
    """The nwant eigenpairs of K x = mu M x nearest sigma.

    solve(b) returns (K - sigma M)^{-1} b.  v1: start vector (length N).
    Returns (mu sorted by |mu - sigma|, X (nwant x N, M-orthonormal columns),
    number of restarts, operator applications)."""
    N = M.shape[0]
    if not 0 < nwant < m <= N:
        raise ValueError("need 0 < nwant < m <= N")
    V = np.zeros((N, m + 1))
    T = np.zeros((m + 1, m))
    mnorm = lambda x: float(np.sqrt(x @ (M @ x)))   # noqa: E731
    V[:, 0] = v1 / mnorm(v1)
    k = 0
    n_apply = 0
    for it in range(max_restarts + 1):
        for j in range(k, m):
            r = solve(M @ V[:, j])
            n_apply += 1
            for _ in range(2):                       # full reorthogonalisation
                h = V[:, :j + 1].T @ (M @ r)
                r = r - V[:, :j + 1] @ h
                T[:j + 1, j] += h
            beta = mnorm(r)
            T[j + 1, j] = beta
            V[:, j + 1] = r / beta
        beta = T[m, m - 1]
        Hm = 0.5 * (T[:m, :m] + T[:m, :m].T)        # symmetric up to rounding
        theta, Y = np.linalg.eigh(Hm)
        order = np.argsort(-np.abs(theta))           # |mu - sigma| = 1/|theta|
        est = np.abs(beta * Y[m - 1, :]) / np.abs(theta)
        want = order[:nwant]
        if np.all(est[want] <= tol) or it == max_restarts:
            break
        # thick restart: keep the kk Ritz vectors nearest sigma
        kk = min(nwant + 2, m - 2)
        keep = order[:kk]
        Yk = Y[:, keep]
        V[:, :kk] = V[:, :m] @ Yk
        V[:, kk] = V[:, m]
        Tn = np.zeros((m + 1, m))
        Tn[:kk, :kk] = np.diag(theta[keep])
        Tn[kk, :kk] = beta * Yk[m - 1, :]
        T = Tn
        k = kk
    mu = sigma + 1.0 / theta[want]
    X = (V[:, :m] @ Y[:, want]).T
    return mu, X, it, n_apply, est[want]


def residual(K, M, mu, x):
    """||K x - mu M x|| / ((||K|| + |mu| ||M||) ||x||), max-row-sum norms."""
    nK = abs(K).sum(axis=1).max()
    nM = abs(M).sum(axis=1).max()
    return float(np.linalg.norm(K @ x - mu * (M @ x)) / ((nK + abs(mu) * nM) * np.linalg.norm(x)))


def slice(sym, K, M, a, b, m, v1, tol=1e-10, extra=4):
    """Eigenpairs with mu in [a, b): count = inertia(b) - inertia(a); Lanczos
    at the midpoint for count + extra pairs; those inside the interval are
    returned, certified when there are exactly `count` of them."""
    count = inertia(sym, K, M, b) - inertia(sym, K, M, a)
    if count == 0:
        return np.zeros(0), np.zeros((0, M.shape[0])), 0, True
    sigma = 0.5 * (a + b)
    F = factorize(sym, (K - sigma * M).tocsr(), indefinite=True)
    mu, X, _, _, _ = lanczos(K, M, sigma, min(count + extra, m - 2), m, F.solve, v1, tol=tol)
    inside = (mu >= a) & (mu < b)
    order = np.argsort(mu[inside])
    return mu[inside][order], X[inside][order], count, int(inside.sum()) == count
