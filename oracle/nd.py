"""Separator-induced nested dissection and symbolic factorisation (oracle).

Plain restatement, test infrastructure only.  The paper orders with METIS
(Section 5.1); here the ordering is the canonical geometric one induced by
rIGA's C^0 separators (Section 3.3: the low-continuity hyperplanes coincide
with the separators of the multifrontal solver's partitioning levels).

Canonical rule on a DOF index box [x0,x1) x [y0,y1):

1. a direction is C^0-cuttable when a C^0 DOF line c lies strictly inside it
   (x0 < c < x1 - 1); its cut is the C^0 line nearest (lo + hi - 1)/2, ties
   to the lower index;
2. if both directions are C^0-cuttable the longer one is cut (tie: x);
3. with no C^0 line left (inside a macroelement, or everywhere for IGA) the
   longer direction (tie: x) of extent E is cut by a p-wide separator
   starting at lo + (E - p)//2, provided E > leaf_min and E >= p + 2;
   otherwise the box is a leaf;
4. each box (leaf or separator) lists its DOFs lexicographically, x fastest;
   post-order is low child, high child, separator.

A supernode is the DOF set of one box.  Its structure (update list) is the
exact symbolic union: the later-ordered neighbours of its pivots in the
matrix graph plus its children's structures, less its own pivots.  Its
parent is the supernode holding the first entry of its structure.
"""
import numpy as np


def nd_boxes(n, c0, p, leaf_min=8, use_c0=True):
    """Post-ordered list of boxes (x0, x1, y0, y1) for an n x n DOF grid."""
    c0 = sorted(c0) if use_c0 else []
    out = []

    def rec(x0, x1, y0, y1):
        if x1 <= x0 or y1 <= y0:
            return
        cx = [c for c in c0 if x0 < c < x1 - 1]
        cy = [c for c in c0 if y0 < c < y1 - 1]
        ex, ey = x1 - x0, y1 - y0
        if cx or cy:
            if cx and cy:
                d = 'x' if ex >= ey else 'y'
            else:
                d = 'x' if cx else 'y'
            lo, hi, cs = (x0, x1, cx) if d == 'x' else (y0, y1, cy)
            c = min(cs, key=lambda v: (abs(2 * v - (lo + hi - 1)), v))
            s0, s1 = c, c + 1
        else:
            d = 'x' if ex >= ey else 'y'
            lo, hi = (x0, x1) if d == 'x' else (y0, y1)
            E = hi - lo
            if not (E > leaf_min and E >= p + 2):
                out.append((x0, x1, y0, y1))
                return
            s0 = lo + (E - p) // 2
            s1 = s0 + p
        if d == 'x':
            rec(x0, s0, y0, y1)
            rec(s1, x1, y0, y1)
            out.append((s0, s1, y0, y1))
        else:
            rec(x0, x1, y0, s0)
            rec(x0, x1, s1, y1)
            out.append((x0, x1, s0, s1))

    rec(0, n, 0, n)
    return out


class Symbolic:
    """Ordering, supernodes, assembly tree, structures and level sets."""

    def __init__(self, perm, sptr, parent, upd_ptr, upd_idx, level):
        self.perm = perm            # perm[new] = old DOF id
        self.iperm = np.empty_like(perm)
        self.iperm[perm] = np.arange(len(perm), dtype=perm.dtype)
        self.sptr = sptr            # pivots of s: new ids [sptr[s], sptr[s+1])
        self.parent = parent        # -1 for a root
        self.upd_ptr = upd_ptr      # struct of s: upd_idx[upd_ptr[s]:upd_ptr[s+1]]
        self.upd_idx = upd_idx      # new ids, ascending
        self.level = level          # 0 for leaves, 1 + max(children) otherwise
        self.nsuper = len(sptr) - 1

    def struct(self, s):
        return self.upd_idx[self.upd_ptr[s]:self.upd_ptr[s + 1]]

    def children(self):
        ch = [[] for _ in range(self.nsuper)]
        for s in range(self.nsuper):
            if self.parent[s] >= 0:
                ch[self.parent[s]].append(s)
        return ch

    def nnz_L(self):
        """Entries of the supernodal factor (dense lower pivot blocks): the
        storage a supernodal factorisation holds and its sweeps read."""
        tot = 0
        for s in range(self.nsuper):
            k = int(self.sptr[s + 1] - self.sptr[s])
            u = int(self.upd_ptr[s + 1] - self.upd_ptr[s])
            tot += k * (k + 1) // 2 + k * u
        return tot

    def factor_flops(self):
        """Cholesky flop count sum_j (c_j^2 + 2 c_j), c_j = off-diagonal
        entries of column j in the supernodal structure (dense pivot
        blocks: the work a supernodal factorisation executes)."""
        tot = 0
        for s in range(self.nsuper):
            k = int(self.sptr[s + 1] - self.sptr[s])
            u = int(self.upd_ptr[s + 1] - self.upd_ptr[s])
            for t in range(k):
                c = (k - 1 - t) + u
                tot += c * c + 2 * c
        return tot

    def scalar_col_counts(self, indptr, indices):
        """Exact off-diagonal count c_j of every column of L (new order):
        the textbook column structure with the elimination tree,
        struct(j) = {i > j : Q_ij != 0} union the structures of j's
        etree children less {j}, the etree parent of j being the first
        entry of struct(j).  No supernodal amalgamation: pivot blocks count
        only their structurally non-zero entries."""
        N = len(self.perm)
        kids = [[] for _ in range(N)]
        st = [None] * N
        cnt = np.zeros(N, dtype=np.int64)
        for j in range(N):
            o = self.perm[j]
            nb = self.iperm[indices[indptr[o]:indptr[o + 1]]]
            s = set(int(i) for i in nb if i > j)
            for c in kids[j]:
                s |= st[c]
                st[c] = None
            s.discard(j)
            st[j] = s
            cnt[j] = len(s)
            if s:
                kids[min(s)].append(j)
        return cnt

    def nnz_L_scalar(self, indptr, indices):
        """Structurally non-zero entries of L including the diagonal,
        sum_j (1 + c_j): the algorithmic size of the factor."""
        return int((self.scalar_col_counts(indptr, indices) + 1).sum())

    def factor_flops_scalar(self, indptr, indices):
        """Algorithmic Cholesky flop count sum_j (c_j^2 + 2 c_j) with the
        exact column counts c_j."""
        c = self.scalar_col_counts(indptr, indices)
        return int((c * c + 2 * c).sum())


def symbolic(n, c0, p, indptr, indices, leaf_min=8, use_c0=True):
    """Canonical ND + exact supernodal symbolic factorisation.

    indptr/indices: CSR pattern of the matrix in the original DOF order.
    """
    boxes = nd_boxes(n, c0, p, leaf_min, use_c0)
    perm = []
    sptr = [0]
    for (x0, x1, y0, y1) in boxes:
        for y in range(y0, y1):
            for x in range(x0, x1):
                perm.append(x + n * y)
        sptr.append(len(perm))
    perm = np.array(perm, dtype=np.int64)
    N = n * n
    if len(perm) != N or len(np.unique(perm)) != N:
        raise AssertionError("boxes must partition the DOFs")
    iperm = np.empty(N, dtype=np.int64)
    iperm[perm] = np.arange(N)
    sptr = np.array(sptr, dtype=np.int64)
    ns = len(sptr) - 1
    owner = np.repeat(np.arange(ns), np.diff(sptr))

    parent = np.full(ns, -1, dtype=np.int64)
    children = [[] for _ in range(ns)]
    structs = []
    level = np.zeros(ns, dtype=np.int64)
    for s in range(ns):
        a, b = sptr[s], sptr[s + 1]
        olds = perm[a:b]
        nb = [indices[indptr[o]:indptr[o + 1]] for o in olds]
        cand = [iperm[np.concatenate(nb)]] + [structs[c] for c in children[s]]
        allc = np.unique(np.concatenate(cand))
        st = allc[allc >= b]
        structs.append(st)
        if len(st):
            parent[s] = owner[st[0]]
            children[parent[s]].append(s)
        if children[s]:
            level[s] = 1 + max(level[c] for c in children[s])
    upd_ptr = np.zeros(ns + 1, dtype=np.int64)
    upd_ptr[1:] = np.cumsum([len(x) for x in structs])
    upd_idx = (np.concatenate(structs) if structs else np.zeros(0)).astype(np.int64)
    return Symbolic(perm, sptr, parent, upd_ptr, upd_idx, level)
