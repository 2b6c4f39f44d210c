"""Multifrontal LDL^T factorisation and supernodal forward/backward solves.

Plain FP64 restatement, test infrastructure only.  The paper factorises the
shifted quadratic pencil once (Algorithm 2, "Factorize Q(s)") with the
multifrontal solver MUMPS and reuses the factors in every forward/backward
elimination (Section 4.2.2).  For a real shift sigma > 0 and K, M SPD, C PSD,
Q(sigma) = sigma^2 M + sigma C + K is SPD, so LDL^T without pivoting exists.

Per supernode s in post-order:
  front F (symmetric, index list = pivots of s then struct(s)) =
      original entries of Q in the pivot columns  +  children's update blocks;
  right-looking LDL^T of the k pivot columns, one column at a time:
      d_t = F[t,t];  l = F[t+1:, t] / d_t;  F[t+1:, t+1:] -= d_t l l^T;
  the first k columns are the factor columns of s; F[k:, k:] is the update
  block handed to the parent.
"""
import numpy as np
import scipy.linalg as sla


class PivotError(ArithmeticError):
    pass


class Factor:
    def __init__(self, sym, Lblocks, D):
        self.sym = sym
        self.L = Lblocks   # per supernode: (k+u) x k, unit lower in its top k x k
        self.D = D         # length N, new ordering

    def solve(self, b):
        """x = Q^{-1} b with b, x in the ORIGINAL DOF order.

        Forward:  L11 x_s = x_s (unit lower), x_struct -= L21 x_s, leaves first.
        Diagonal: x /= D.
        Backward: x_s -= L21^T x_struct, L11^T x_s = x_s, root first.
        """
        sym = self.sym
        dt = np.result_type(self.D.dtype, np.asarray(b).dtype)
        x = np.asarray(b, dtype=dt)[sym.perm].copy()
        for s in range(sym.nsuper):
            a, e = sym.sptr[s], sym.sptr[s + 1]
            k = e - a
            L = self.L[s]
            x[a:e] = sla.solve_triangular(L[:k], x[a:e], lower=True, unit_diagonal=True)
            st = sym.struct(s)
            if len(st):
                x[st] -= L[k:] @ x[a:e]
        x /= self.D
        for s in range(sym.nsuper - 1, -1, -1):
            a, e = sym.sptr[s], sym.sptr[s + 1]
            k = e - a
            L = self.L[s]
            st = sym.struct(s)
            if len(st):
                x[a:e] -= L[k:].T @ x[st]
            x[a:e] = sla.solve_triangular(L[:k], x[a:e], lower=True, unit_diagonal=True,
                                          trans='T')
        out = np.empty_like(x)
        out[sym.perm] = x
        return out


def factorize(sym, Q, indefinite=False):
    """Multifrontal LDL^T of the symmetric CSR matrix Q (original order).

    indefinite=False: Q must be positive definite (a non-positive pivot
    raises PivotError).  indefinite=True: pivots of either sign are kept (a
    zero or non-finite pivot raises), as for Q = K - mu M with mu inside the
    spectrum (spectrum slicing, Section 4.1.4); D then carries the inertia."""
    Q = Q.tocsr()
    N = Q.shape[0]
    ns = sym.nsuper
    children = sym.children()
    Lblocks = [None] * ns
    cplx = np.iscomplexobj(Q.data)
    dt = np.complex128 if cplx else np.float64
    D = np.zeros(N, dtype=dt)
    upd = [None] * ns
    for s in range(ns):
        a, e = int(sym.sptr[s]), int(sym.sptr[s + 1])
        k = e - a
        st = sym.struct(s)
        idx = np.concatenate([np.arange(a, e), st])
        F = np.zeros((len(idx), len(idx)), dtype=dt)
        # original entries of the pivot columns (symmetric: both triangles)
        for t in range(k):
            old = sym.perm[a + t]
            cols = sym.iperm[Q.indices[Q.indptr[old]:Q.indptr[old + 1]]]
            vals = Q.data[Q.indptr[old]:Q.indptr[old + 1]]
            for i, v in zip(cols, vals):
                if i < a + t:
                    continue          # upper triangle in the new order
                pi = int(i - a) if i < e else k + int(np.searchsorted(st, i))
                if pi >= k and (pi - k >= len(st) or st[pi - k] != i):
                    raise AssertionError("entry outside the front structure")
                F[pi, t] += v
                if pi != t:
                    F[t, pi] += v
        # extend-add of the children's update blocks
        for c in children[s]:
            sc = sym.struct(c)
            rm = np.where(sc < e, sc - a, k + np.searchsorted(st, sc))
            F[np.ix_(rm, rm)] += upd[c]
            upd[c] = None
        # partial LDL^T of the k pivot columns
        for t in range(k):
            d = F[t, t]
            if cplx:   # complex symmetric (unconjugated) LDL^T
                if not (d != 0.0 and np.isfinite(d)):
                    raise PivotError(f"zero pivot at supernode {s}")
            elif indefinite:
                if not (d != 0.0 and np.isfinite(d)):
                    raise PivotError(f"zero pivot at supernode {s}")
            elif not d > 0.0:
                raise PivotError(f"non-positive pivot {d} at supernode {s}")
            l = F[t + 1:, t] / d
            F[t + 1:, t + 1:] -= d * np.outer(l, l)
            F[t + 1:, t] = l
            F[t, t + 1:] = 0.0
            F[t, t] = 1.0
            D[a + t] = d
        Lblocks[s] = F[:, :k].copy()
        upd[s] = F[k:, k:].copy()
    return Factor(sym, Lblocks, D)
