"""Matrix size and pattern counts of B-spline discretisations (oracle).

Test infrastructure only.  Used to pin the knot-multiplicity and support
logic of ``bspline`` against the sizes the paper prints for its Fig. 4
(64 x 64 elements, p = 4, H(curl) IGA versus rIGA with 16 x 16-element
macroelements, Section 3.3).

H(curl) space, Section 3.2 / 3.3: S^{p-1,p} x S^{p,p-1} (x and y components).
In rIGA both univariate factors get multiplicity p-1 at the macroelement
boundaries (C^0 for the degree p-1 factor, C^1 for the degree p factor).
No boundary condition is imposed for this count.  The pattern of K u M is the
union of the four component blocks; a block's entry count is the product of
the univariate coupled-pair counts in xi and eta, two functions being coupled
when their supports share an open interval.
"""
from .bspline import knot_vector, n_functions, coupled


def pair_count(ka, pa, kb, pb):
    """Number of coupled (i, j) pairs between two univariate spaces."""
    na, nb = n_functions(ka, pa), n_functions(kb, pb)
    tot = 0
    for i in range(na):
        a0, a1 = ka[i], ka[i + pa + 1]
        for j in range(nb):
            b0, b1 = kb[j], kb[j + pb + 1]
            if max(a0, b0) < min(a1, b1):
                tot += 1
    return tot


def hcurl_counts(ne, p, block=0):
    """(N, nnz) of the H(curl) matrix pattern, IGA (block=0) or rIGA."""
    kp = knot_vector(ne, p, block, sep_mult=p - 1)
    kq = knot_vector(ne, p - 1, block, sep_mult=p - 1)
    n_p, n_q = n_functions(kp, p), n_functions(kq, p - 1)
    # x component: degree p-1 in xi, p in eta; y component: p in xi, p-1 in eta
    N = n_q * n_p + n_p * n_q
    qq = pair_count(kq, p - 1, kq, p - 1)
    pp = pair_count(kp, p, kp, p)
    qp = pair_count(kq, p - 1, kp, p)
    nnz = qq * pp + pp * qq + 2 * qp * qp
    return N, nnz


def h1_counts(ne, p, block=0):
    """(N, nnz) of the scalar H^1 pattern with Dirichlet functions removed."""
    k = knot_vector(ne, p, block)
    nf = n_functions(k, p)
    pairs = 0
    for i in range(1, nf - 1):
        for j in range(1, nf - 1):
            if coupled(k, p, i, j):
                pairs += 1
    return (nf - 2) ** 2, pairs * pairs
