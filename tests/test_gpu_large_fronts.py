"""Factorisations with pivot blocks wider than 256 pivots.

Those blocks are factorised and inverted by the blocked multi-CTA kernels
(k_wide_*).  The maximum-continuity space (block 0) has them from ne = 96:
at ne = 128 and 192 (p = 3) the real and complex solves are compared with
the oracle's factorisation entry by entry.  At ne = 320 the top pivot block
has 963 pivots, so the complex factor's row panels (16 rows x 963 complex
entries, 246 KB) also go through the global buffer instead of shared
memory; those solves are checked by their normwise backward error against
the library's own exported K, M, C (the oracle's Python factorisation of
this 103,041-DOF system would take minutes).
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle.assemble import assemble
from oracle.multifrontal import factorize
from oracle.nd import symbolic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NE, P, BLOCK = 320, 3, 0


@pytest.fixture(scope="module")
def rq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_14064_gb300 import build, rigaqep
    build.build()
    rigaqep.load()
    return rigaqep


@pytest.fixture(scope="module")
def problem(rq):
    rng = np.random.default_rng(20211234)
    sig = rng.uniform(0.1, 1.0, NE * NE)
    pr = rq.Problem(NE, P, BLOCK, sig).analyze()
    sym = pr.export_symbolic()
    assert np.diff(sym["sptr"]).max() > 800   # the path under test
    csr = pr.export_csr()
    shape = (pr.N, pr.N)
    mats = {k: sp.csr_matrix((csr[k], csr["col"], csr["rowptr"]), shape=shape)
            for k in ("K", "M", "C")}
    yield pr, mats
    pr.close()


def _backward_error(Q, x, b):
    nQ = abs(Q).sum(axis=1).max()
    return np.linalg.norm(Q @ x - b, np.inf) / (nQ * np.linalg.norm(x, np.inf) + np.linalg.norm(b, np.inf))


def test_real_factor_with_wide_pivot_block(problem):
    pr, A = problem
    sigma = 7.5
    pr.factor(sigma)
    b = np.random.default_rng(1).standard_normal(pr.N)
    x = pr.solve(torch.from_numpy(b).cuda()).cpu().numpy()
    Q = (A["K"] + sigma * A["C"] + sigma * sigma * A["M"]).tocsr()
    assert _backward_error(Q, x, b) <= 1e-13


def test_complex_factor_with_global_row_panels(problem):
    pr, A = problem
    s = 2.0 + 25.0j
    pr.factor_complex(s)
    rng = np.random.default_rng(2)
    b = rng.standard_normal(pr.N) + 1j * rng.standard_normal(pr.N)
    x = pr.solve_complex(torch.from_numpy(b).cuda()).cpu().numpy()
    Q = (A["K"] + s * A["C"] + s * s * A["M"]).tocsr()
    assert _backward_error(Q, x, b) <= 1e-13


@pytest.mark.parametrize("ne,shift", [(192, 3.0), (128, 2.0 + 20.0j)])
def test_wide_pivot_blocks_match_oracle(rq, ne, shift):
    rng = np.random.default_rng(ne)
    sig = rng.uniform(0.1, 1.0, ne * ne)
    A = assemble(ne, P, BLOCK, sig)
    sym = symbolic(A.n1, A.space.c0_dofs, P, A.indptr, A.indices, use_c0=False)
    Q = (A.K + shift * A.C + shift * shift * A.M).tocsr()
    F = factorize(sym, Q)
    cplx = isinstance(shift, complex)
    b = rng.standard_normal(A.N) + (1j * rng.standard_normal(A.N) if cplx else 0.0)
    ref = F.solve(b)
    pr = rq.Problem(ne, P, BLOCK, sig).analyze()
    assert np.diff(pr.export_symbolic()["sptr"]).max() > 256   # the path under test
    if cplx:
        x = pr.factor_complex(shift).solve_complex(torch.from_numpy(b).cuda()).cpu().numpy()
    else:
        x = pr.factor(shift).solve(torch.from_numpy(b).cuda()).cpu().numpy()
    assert np.abs(x - ref).max() <= 1e-11 * np.abs(ref).max()
    pr.close()
