"""Multiset comparison of computed eigenvalues with a reference list.

Repeated eigenvalues (x <-> y mirror symmetry of a mesh with constant
damping gives exact doubles) must be matched by as many distinct copies:
each computed value is assigned to its own reference value, never two
computed values to one reference value.  The comparison is the bottleneck
assignment: the smallest t such that a one-to-one assignment exists with
every relative distance |ref - got| / |got| <= t.
"""
import numpy as np
from scipy.optimize import linear_sum_assignment


def _feasible(cost, t):
    """A one-to-one assignment of every row to a distinct column with
    cost <= t exists (maximum bipartite matching via a 0/1 assignment)."""
    miss = (cost > t).astype(np.float64)
    r, c = linear_sum_assignment(miss)
    return miss[r, c].sum() == 0.0


def multiset_max_rel(ref, got):
    """Bottleneck relative distance of a one-to-one assignment of the values
    `got` to distinct values of `ref` (len(ref) >= len(got))."""
    ref = np.asarray(ref, dtype=np.complex128).ravel()
    got = np.asarray(got, dtype=np.complex128).ravel()
    if len(got) == 0:
        return 0.0
    if len(ref) < len(got):
        return float("inf")
    cost = np.abs(got[:, None] - ref[None, :]) / np.abs(got)[:, None]
    levels = np.unique(cost)
    lo, hi = 0, len(levels) - 1
    while lo < hi:                       # smallest feasible threshold
        mid = (lo + hi) // 2
        if _feasible(cost, levels[mid]):
            hi = mid
        else:
            lo = mid + 1
    return float(levels[lo])


def same_multiset(a, b, rtol):
    """a and b have equal length and match one to one within rtol."""
    return len(a) == len(b) and multiset_max_rel(a, b) <= rtol
