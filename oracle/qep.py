"""Shift-and-invert Krylov--Schur solve of the linearised QEP (oracle).

Plain FP64 restatement, test infrastructure only.

* Linearisation, Eq. (Linearization): A = [[0, I], [-K, -C]], B = diag(I, M),
  eigenvector [u; lambda u].
* Operator, Eq. (BlockOperatorVector): r = L(s)^{-1} B v with
      r_u = -Q(s)^{-1} (s M v_u + C v_u + M v_l),   r_l = s r_u + v_u.
* B-inner product, Section 4.2.1: <x, y>_B = x_u^T y_u + x_l^T M y_l.
* Arnoldi recurrence, Algorithm 1 / Algorithm 2: h = V^T B r, z = r - V h,
  h_{j+1,j} = ||z||_B; classical Gram--Schmidt applied twice (CGS2).
* Rayleigh--Ritz, Eq. (ArnoldiRitz): Ritz values theta of the projected
  matrix; lambda = s + 1/theta (Section 4.1.1, theta = 1/(lambda - s)).
* Restart: Krylov--Schur (Section 4.1.3; the paper omits the details, this is
  Stewart's scheme): real Schur form of the projected matrix, wanted Ritz
  values moved to the top, the first k Schur vectors kept; converged kept
  Ritz values are locked (moved to the front, their spike entries dropped).

Readings where the paper is silent:
* wanted set = the neig Ritz values nearest s; for equal distances Im > 0
  first (conjugate pairs tie exactly for a real shift);
* k = ncand + 2 kept (at most m - 2, at least ncand), plus one when that would
  split a conjugate pair;
* a Ritz pair is converged when |h_{m+1,m} y_m| / |theta| <= tol (y unit);
* the QEP eigenvector is the upper block x = V_u y, scaled to unit 2-norm with
  its largest-modulus entry real and positive (lowest index on ties);
* the reported accuracy is the normwise backward error
  eta = ||Q(lambda) x|| / ((|lambda|^2 ||M|| + |lambda| ||C|| + ||K||) ||x||)
  with max-row-sum norms for the matrices.

Target/shift split (the paper places its single shift inside the spectrum
region of interest, Section 4.1.4): with a target t different from the shift
s, the ncand pairs nearest s are converged and the neig of them nearest t are
returned.  The choice is certified when no unconverged eigenvalue can be
nearer t, under one assumption the Krylov iteration does not prove: that
every eigenvalue within r of s (r the largest candidate distance) is among
the candidates (Krylov--Schur converges the eigenvalues nearest the shift
first).  Given that, for K, M SPD and C = sum sigma_e M_e with
sigma_e >= 0, x^H(lambda^2 M + lambda C + K)x = 0 gives complex eigenvalues
Re lambda = -x^H C x / (2 x^H M x) <= -min(sigma_e)/2 and real ones <= 0, so
for 0 <= s <= t
  complex: |lambda - t|^2 >= r^2 + (t - s)(t + s + min sigma_e),
  real:    |lambda - t|   >= (t - s) + r.
"""
import numpy as np
import scipy.linalg as sla
from scipy.linalg import lapack


def apply_operator(v, s, M, C, solve):
    """Eq. (BlockOperatorVector)."""
    N = M.shape[0]
    vu, vl = v[:N], v[N:]
    ru = -solve(s * (M @ vu) + C @ vu + M @ vl)
    return np.concatenate([ru, s * ru + vu])


def b_apply(x, M):
    """B x = [x_u; M x_l]."""
    N = M.shape[0]
    return np.concatenate([x[:N], M @ x[N:]])


def b_norm(x, M):
    return float(np.sqrt(x @ b_apply(x, M)))


def wanted_order(lam, s):
    """Indices of lam sorted by |lam - s|, Im > 0 first on ties."""
    key_d = np.abs(lam - s)
    key_i = np.where(lam.imag > 0, 0, np.where(lam.imag == 0, 1, 2))
    return np.lexsort((key_i, key_d))


def normalise_vector(x):
    """Unit 2-norm, largest-modulus entry real positive (lowest index on ties)."""
    x = x / np.linalg.norm(x)
    a = np.abs(x)
    i = int(np.flatnonzero(a == a.max())[0])
    return x * (np.conj(x[i]) / a[i])


def backward_error(lam, x, K, C, M):
    nK = abs(K).sum(axis=1).max()
    nC = abs(C).sum(axis=1).max()
    nM = abs(M).sum(axis=1).max()
    r = K @ x + lam * (C @ x) + lam * lam * (M @ x)
    den = (abs(lam) ** 2 * nM + abs(lam) * nC + nK) * np.linalg.norm(x)
    return float(np.linalg.norm(r) / den)


class EigsResult:
    def __init__(self, lam, X, eta, n_conv, n_restarts, n_apply, n_vv):
        self.lam, self.X, self.eta = lam, X, eta
        self.n_conv, self.n_restarts, self.n_apply = n_conv, n_restarts, n_apply
        self.n_vv = n_vv


def eigs(K, C, M, s, neig, m, solve, v1, tol=1e-10, max_restarts=1000, target=None,
         ncand=None, sigma_min=None, op=None):
    """Algorithm 2 with CGS2 and Krylov--Schur restarts.

    solve(b) must return Q(s)^{-1} b (the factorised shifted pencil).
    v1: start vector of length 2N (original DOF order).
    target/ncand/sigma_min: the target/shift split described above (target
    None: the shift is the target and ncand = neig).
    op: another operator on 2N vectors in place of Eq. (BlockOperatorVector)
    (the complex-shift real operator); lambda is then s + 1/theta of its
    Ritz values theta (see eigs_complex_shift).
    """
    N = M.shape[0]
    ncand = neig if ncand is None else ncand
    if not (0 < neig <= ncand < m <= 2 * N):
        raise ValueError("need 0 < neig <= ncand < m <= 2N")
    V = np.zeros((2 * N, m + 1))
    H = np.zeros((m + 1, m))
    V[:, 0] = v1 / b_norm(v1, M)
    k = 0
    lock = 0        # leading Schur columns locked (converged, decoupled)
    n_apply = 0
    n_vv = 0
    steps = []      # basis index j of every operator application, in order
    for it in range(max_restarts + 1):
        for j in range(k, m):
            r = apply_operator(V[:, j], s, M, C, solve) if op is None else op(V[:, j])
            n_apply += 1
            steps.append(j)
            for _ in range(2):                      # CGS2
                h = V[:, :j + 1].T @ b_apply(r, M)
                r = r - V[:, :j + 1] @ h
                H[:j + 1, j] += h
                n_vv += 2 * (j + 1)
            nr = b_norm(r, M)
            H[j + 1, j] = nr
            V[:, j + 1] = r / nr
        Hm = H[:m, :m]
        beta = H[m, m - 1]
        theta, Y = np.linalg.eig(Hm)          # Ritz pairs, unit columns
        lam = s + 1.0 / theta
        order = wanted_order(lam, s)
        est = np.abs(beta * Y[m - 1, :]) / np.abs(theta)
        want = order[:ncand]
        conv = est[want] <= tol
        if conv.all() or it == max_restarts:
            break
        T, Z = sla.schur(Hm, output='real')
        wr, wi = _schur_eigs(T)
        order = wanted_order(s + 1.0 / (wr + 1j * wi), s)
        kk = min(ncand + 2, max(ncand, m - 2))
        sel_idx = set(order[:kk].tolist()) | set(range(lock))
        # keep conjugate partners together
        pos = 0
        while pos < m:
            if pos + 1 < m and T[pos + 1, pos] != 0.0:
                if pos in sel_idx or pos + 1 in sel_idx:
                    sel_idx |= {pos, pos + 1}
                pos += 2
            else:
                pos += 1
        select = np.zeros(m, dtype=np.int32)
        select[list(sel_idx)] = 1
        T2, Z2, info = _trsen(select, T, Z)
        k = int(select.sum())
        # locking: converged kept Ritz values move to the front and their
        # spike entries are dropped (decoupled from the active part)
        conv_pos = _converged_positions(T2, theta, est, want, tol, k)
        conv_pos[:lock] = 1
        T3, Z3, info = _trsen(conv_pos.astype(np.int32), T2, Z2)
        lock = int(conv_pos.sum())
        V[:, :k] = V[:, :m] @ Z3[:, :k]
        V[:, k] = V[:, m]
        Hn = np.zeros((m + 1, m))
        Hn[:k, :k] = T3[:k, :k]
        Hn[k, lock:k] = beta * Z3[m - 1, lock:k]
        H = Hn
    cand = want
    lam_c = lam[cand]
    certified = bool(conv.all())
    if target is None:
        chosen = np.arange(neig)
    else:
        chosen = wanted_order(lam_c, target)[:neig]
        dmax = np.abs(lam_c[chosen] - target).max()
        r = np.abs(lam_c - s).max()
        ok = (certified and s >= 0 and target >= s and sigma_min is not None
              and sigma_min >= 0)
        if ok:
            bound = min(np.sqrt(r * r + (target - s) * (target + s + sigma_min)),
                        (target - s) + r)
            certified = bool(bound >= dmax * (1 + 1e-12))
        else:
            certified = False
    X = []
    eta = []
    lam_w = lam_c[chosen]
    for t, i in enumerate(np.asarray(cand)[chosen]):
        x = normalise_vector(V[:N, :m] @ Y[:, i])
        X.append(x)
        eta.append(backward_error(lam_w[t], x, K, C, M))
    res = EigsResult(lam_w, np.array(X), np.array(eta), int(conv[chosen].sum()), it,
                     n_apply, n_vv)
    res.certified = certified
    res.candidates = lam_c        # the ncand converged values around the shift
    res.steps = steps
    return res


def _converged_positions(T, theta, est, want, tol, k):
    """1 at the Schur positions < k holding a converged wanted Ritz value
    (matched to the eigenvalues of the projected matrix by nearest value);
    conjugate pairs are flagged together."""
    wr, wi = _schur_eigs(T)
    m = T.shape[0]
    flags = np.zeros(m, dtype=np.int64)
    good = [i for i in want if est[i] <= tol]
    for pos in range(k):
        z = wr[pos] + 1j * wi[pos]
        j = int(np.argmin(np.abs(theta - z)))
        if j in good and abs(theta[j] - z) <= 1e-8 * abs(z):
            flags[pos] = 1
    pos = 0
    while pos < k:
        if pos + 1 < m and T[pos + 1, pos] != 0.0:
            f = flags[pos] & flags[pos + 1]
            flags[pos] = flags[pos + 1] = f
            pos += 2
        else:
            pos += 1
    return flags


def _schur_eigs(T):
    m = T.shape[0]
    wr = np.zeros(m)
    wi = np.zeros(m)
    pos = 0
    while pos < m:
        if pos + 1 < m and T[pos + 1, pos] != 0.0:
            a, b, c, d = T[pos, pos], T[pos, pos + 1], T[pos + 1, pos], T[pos + 1, pos + 1]
            ev = np.linalg.eigvals(np.array([[a, b], [c, d]]))
            ev = ev[np.argsort(-ev.imag)]
            wr[pos], wi[pos] = ev[0].real, ev[0].imag
            wr[pos + 1], wi[pos + 1] = ev[1].real, ev[1].imag
            pos += 2
        else:
            wr[pos] = T[pos, pos]
            pos += 1
    return wr, wi


def _trsen(select, T, Z):
    out = lapack.dtrsen(select, T, Z, job='N')
    T2, Z2 = out[0], out[1]
    info = out[-1]
    if info != 0:
        raise ArithmeticError(f"dtrsen failed: {info}")
    return T2, Z2, info


def scaling_factor(K, M):
    """Remark 4: varsigma = sqrt(||K|| / ||M||) with the paper's "infinity
    norm", the largest absolute entry of the matrix."""
    return float(np.sqrt(abs(K).max() / abs(M).max()))


def eigs_scaled(K, C, M, s, neig, m, solve, v1, tol=1e-10, max_restarts=1000, target=None,
                ncand=None, sigma_min=None):
    """The scaled eigenproblem of Remark 4: (K + gamma C_s + gamma^2 M_s) u = 0
    with C_s = varsigma C, M_s = varsigma^2 M and gamma = lambda / varsigma.
    Its shifted matrix at gamma_s = s / varsigma is Q(s) itself, so the same
    solve serves; the target and the damping bound scale like gamma.  The
    result is mapped back to lambda = varsigma gamma (eigenvectors u are
    shared; backward errors are those of the original QEP)."""
    vs = scaling_factor(K, M)
    r = eigs(K, vs * C, vs * vs * M, s / vs, neig, m, solve, v1, tol=tol,
             max_restarts=max_restarts, target=None if target is None else target / vs,
             ncand=ncand, sigma_min=None if sigma_min is None else sigma_min / vs)
    r.lam = vs * r.lam
    r.candidates = vs * r.candidates
    r.eta = np.array([backward_error(l, x, K, C, M) for l, x in zip(r.lam, r.X)])
    r.scale = vs
    return r


def eigs_complex_shift(K, C, M, s, neig, m, solve, v1, ncand=None, tol=1e-10,
                       max_restarts=1000):
    """Eigenpairs nearest a complex shift s (Section 4.1.1 lets s lie in C).

    solve(b) returns Q(s)^{-1} b for complex b (the complex symmetric factor).
    The recurrence runs on the real operator
        R v = Re(L(s)^{-1} B v) = ((A - s B)^{-1} + (A - conj(s) B)^{-1}) B v / 2
    (Parlett and Saad's real form of a complex shift-and-invert), whose
    eigenvalue for an eigenvalue lambda of the pencil is
        psi = (1/(lambda - s) + 1/(lambda - conj s)) / 2
            = (lambda - a) / ((lambda - s)(lambda - conj s)),  a = Re s.
    The ncand Ritz values of largest modulus (eigenvalues nearest s or conj s)
    are converged; each gives the two roots of
        psi l^2 - (2 a psi + 1) l + psi |s|^2 + a = 0,
    of which the one with the smaller backward error (same eigenvector
    x = V_u y) is the eigenvalue.  The neig nearest s are returned."""
    ncand = 2 * neig + 4 if ncand is None else ncand
    op = lambda v: np.real(apply_operator(v.astype(complex), s, M, C, solve))  # noqa: E731
    r = eigs(K, C, M, 0.0, ncand, m, solve, v1, tol=tol, max_restarts=max_restarts, op=op)
    a, s2 = s.real, abs(s) ** 2
    lam, eta = [], []
    for theta_inv, x in zip(r.lam, r.X):
        psi = 1.0 / theta_inv
        roots = np.roots([psi, -(2 * a * psi + 1), psi * s2 + a])
        errs = [backward_error(l, x, K, C, M) for l in roots]
        j = int(np.argmin(errs))
        lam.append(roots[j])
        eta.append(errs[j])
    lam, eta = np.array(lam), np.array(eta)
    order = np.lexsort((-lam.imag, np.abs(lam - s)))[:neig]
    out = EigsResult(lam[order], r.X[order], eta[order], r.n_conv, r.n_restarts, r.n_apply,
                     r.n_vv)
    out.certified = False
    return out
