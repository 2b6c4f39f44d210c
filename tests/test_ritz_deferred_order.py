"""Host check of the ordering argument behind the Ritz step's helper CTAs.

The device QR iteration (csrc/ritz.cu) updates only the active window of T
during a Francis sweep and hands the sweep's reflectors, plus the rotations
of the 2 x 2 blocks standardised before it, to helper CTAs that apply them to
the rest of T and to Z one or two sweeps later.  That is correct because an
entry outside one sweep's window is outside every later window, and the
deflation tests read only diagonal and subdiagonal entries.

This test replays the same sweep structure (chains of up to four double-shift
bulges, four rows apart, in (round, bulge) order) in NumPy with the helper
work delayed by 0 to 3 batches, and checks that
  * no window ever contains an entry that pending helper work touches,
  * T and Z come out bit for bit the same for every delay,
  * the result is a real Schur decomposition of the input.
It checks the argument, not the CUDA code (the GPU tests do that).
"""
import numpy as np
import pytest
import scipy.linalg as sla

EPS = 2.220446049250313e-16


def _refl(x0, x1, x2, n):
    sg = x1 * x1 + (x2 * x2 if n == 3 else 0.0)
    if sg == 0.0:
        return None
    nr = np.sqrt(x0 * x0 + sg)
    beta = nr if x0 <= 0 else -nr
    return (x0 - beta, x1, x2 if n == 3 else 0.0, 1.0 / (beta * (beta - x0)), n)


def _rows(A, r, pos, rows):      # right-multiply columns pos.. of the given rows
    u0, u1, u2, tau, n = r
    for i in rows:
        s = u0 * A[i, pos] + u1 * A[i, pos + 1] + (u2 * A[i, pos + 2] if n == 3 else 0.0)
        s *= tau
        A[i, pos] -= s * u0
        A[i, pos + 1] -= s * u1
        if n == 3:
            A[i, pos + 2] -= s * u2


def _cols(A, r, pos, cols):      # left-multiply rows pos.. of the given columns
    u0, u1, u2, tau, n = r
    for c in cols:
        s = u0 * A[pos, c] + u1 * A[pos + 1, c] + (u2 * A[pos + 2, c] if n == 3 else 0.0)
        s *= tau
        A[pos, c] -= s * u0
        A[pos + 1, c] -= s * u1
        if n == 3:
            A[pos + 2, c] -= s * u2


def _rot(A, ia, ib, c, s):
    a, b = A[ia], A[ib]
    A[ia] = c * a + s * b
    A[ib] = -s * a + c * b


def _std2(T, j):
    a, b, e, d = T[j, j], T[j, j + 1], T[j + 1, j], T[j + 1, j + 1]
    if e == 0.0:
        return None
    hp = 0.5 * (a - d)
    disc = hp * hp + b * e
    if disc >= 0:
        rt = np.sqrt(disc)
        l1 = 0.5 * (a + d) + (rt if hp >= 0 else -rt)
        x1, y1, x2, y2 = b, l1 - a, l1 - d, e
        x, y = (x1, y1) if x1 * x1 + y1 * y1 >= x2 * x2 + y2 * y2 else (x2, y2)
        rn = 1.0 / np.sqrt(x * x + y * y)
        return x * rn, y * rn, False
    pp, qq = -(a - d), b + e
    r2 = pp * pp + qq * qq
    if r2 == 0:
        return 1.0, 0.0, True
    rr = 1.0 / np.sqrt(r2)
    c2, s2 = qq * rr, pp * rr
    if c2 >= 0:
        c = np.sqrt(0.5 * (1 + c2))
        s = s2 * 0.5 / c
    else:
        s = np.sqrt(0.5 * (1 - c2))
        s = -s if s2 < 0 else s
        c = s2 * 0.5 / s
    return c, s, True


def _schur(H, delay, split, nbmax=4, gap=4):
    """Multi-bulge Francis QR of the Hessenberg H.  split=False applies the
    work outside the window right after each sweep; split=True hands it over
    in batches applied `delay` batches late."""
    T = H.copy()
    m = T.shape[0]
    Z = np.eye(m)
    tn = np.linalg.norm(T)
    queue = []
    touched = np.zeros((m, m), bool)

    def helper(batch):
        rots, sweep = batch
        for j, c, s in rots:
            for col in range(j + 2, m):
                _rot(T, (j, col), (j + 1, col), c, s)
                touched[j, col] = touched[j + 1, col] = True
            for r in range(j):
                _rot(T, (r, j), (r, j + 1), c, s)
                touched[r, j] = touched[r, j + 1] = True
            for r in range(m):
                _rot(Z, (r, j), (r, j + 1), c, s)
        if sweep:
            l, hi, refls = sweep
            for r, pos in refls:
                if r is None:
                    continue
                _cols(T, r, pos, range(hi + 1, m))
                touched[pos:pos + r[4], hi + 1:] = True
                _rows(T, r, pos, range(l))
                touched[:l, pos:pos + r[4]] = True
                _rows(Z, r, pos, range(m))

    def publish(batch):
        queue.append(batch)
        while len(queue) > delay:
            helper(queue.pop(0))

    hi, its, rots, sweeps = m - 1, 0, [], 0
    while hi >= 0:
        l = hi
        while l > 0:
            sc = abs(T[l - 1, l - 1]) + abs(T[l, l]) or tn
            if abs(T[l, l - 1]) <= EPS * sc:
                break
            l -= 1
        if l > 0:
            T[l, l - 1] = 0.0
        if l == hi:
            hi, its = hi - 1, 0
            continue
        if l == hi - 1:
            j = hi - 1
            st = _std2(T, j)
            if st is not None:
                c, s, cplx = st
                if split:
                    for col in (j, j + 1):
                        _rot(T, (j, col), (j + 1, col), c, s)
                    for r in (j, j + 1):
                        _rot(T, (r, j), (r, j + 1), c, s)
                    rots.append((j, c, s))
                else:
                    for col in range(j, m):
                        _rot(T, (j, col), (j + 1, col), c, s)
                    for r in range(j + 2):
                        _rot(T, (r, j), (r, j + 1), c, s)
                    for r in range(m):
                        _rot(Z, (r, j), (r, j + 1), c, s)
                if not cplx:
                    T[j + 1, j] = 0.0
                else:
                    T[j, j] = T[j + 1, j + 1] = 0.5 * (T[j, j] + T[j + 1, j + 1])
            hi, its = hi - 2, 0
            continue
        sweeps += 1
        assert sweeps <= 40 * m
        its += 1
        nb = max(1, min(nbmax, (hi - l + 1) // (gap + 2)))
        p = hi - 1
        shifts = []
        for w in range(nb):
            if w == 0 and its % 11 == 10:
                ww = abs(T[hi, hi - 1]) + abs(T[hi - 1, hi - 2])
                z0 = T[hi, hi] + 0.75 * ww
                shifts.append((2 * z0, z0 * z0 + 0.4375 * ww * ww))
            else:
                shifts.append((T[p, p] + T[p + 1, p + 1],
                               T[p, p] * T[p + 1, p + 1] - T[p, p + 1] * T[p + 1, p]))
        if split:   # the window holds nothing that pending helper work touches
            assert not touched[l:hi + 1, l:hi + 1].any()
        refls = []
        for t in range((hi - 1 - l) + gap * (nb - 1) + 1):
            cur = []
            for w in range(nb):
                kq = l + t - gap * w
                if not l <= kq <= hi - 1:
                    cur.append((None, kq))
                    continue
                n = 3 if kq <= hi - 2 else 2
                sh, th = shifts[w]
                if kq == l:
                    x = T[l, l] ** 2 + T[l, l + 1] * T[l + 1, l] - sh * T[l, l] + th
                    y = T[l + 1, l] * (T[l, l] + T[l + 1, l + 1] - sh)
                    z = T[l + 1, l] * T[l + 2, l + 1] if n == 3 else 0.0
                else:
                    x, y = T[kq, kq - 1], T[kq + 1, kq - 1]
                    z = T[kq + 2, kq - 1] if n == 3 else 0.0
                r = _refl(x, y, z, n)
                cur.append((r, kq))
                if r is not None:
                    _rows(T, r, kq, range(l, min(kq + 3, hi) + 1))
            for r, kq in cur:
                if not l <= kq <= hi - 1:
                    continue
                if r is not None:
                    _cols(T, r, kq, range(kq - 1 if kq > l else l, hi + 1))
                if kq > l:
                    T[kq + 1, kq - 1] = 0.0
                    if r is not None and r[4] == 3:
                        T[kq + 2, kq - 1] = 0.0
            refls += cur
        if split:
            publish((rots, (l, hi, refls)))
            rots = []
        else:
            helper(([], (l, hi, refls)))
    if split:
        publish((rots, None))
        while queue:
            helper(queue.pop(0))
    return T, Z


def _matrices():
    rng = np.random.default_rng(20211214)
    yield sla.hessenberg(rng.standard_normal((40, 40)))
    # clustered complex pairs and a graded spectrum, as shift-invert Ritz
    # values of a damped problem
    m = 36
    ev = []
    for k in range(m // 2):
        r = 10.0 ** (-k / 6)
        ev += [r * np.exp(1j * (0.3 + 0.02 * k)), r * np.exp(-1j * (0.3 + 0.02 * k))]
    D = np.zeros((m, m))
    for k in range(m // 2):
        a, b = ev[2 * k].real, ev[2 * k].imag
        D[2 * k:2 * k + 2, 2 * k:2 * k + 2] = [[a, b], [-b, a]]
    Q, _ = np.linalg.qr(rng.standard_normal((m, m)))
    yield sla.hessenberg(Q @ D @ Q.T)


@pytest.mark.parametrize("H", list(_matrices()), ids=["random40", "graded36"])
def test_delayed_helper_work_gives_the_same_schur_form(H):
    T0, Z0 = _schur(H, 0, False)
    for delay in (1, 2, 3):
        T1, Z1 = _schur(H, delay, True)
        assert np.array_equal(T0, T1) and np.array_equal(Z0, Z1), delay
    m = H.shape[0]
    assert np.abs(Z0.T @ Z0 - np.eye(m)).max() < 1e-13
    assert np.abs(Z0 @ T0 @ Z0.T - H).max() < 1e-12 * np.abs(H).max()
    assert np.all(np.abs(np.diag(T0, -1)[1:] * np.diag(T0, -1)[:-1]) == 0.0)   # quasi-triangular
