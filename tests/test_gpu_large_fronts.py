"""Factorisations whose pivot blocks are wider than the cluster kernel's 800.

The maximum-continuity space (block 0) at ne = 320, p = 3 has a top pivot
block of 963 pivots: the real factor takes the one-CTA pivot kernel, and the
complex factor's row panels (16 rows x 963 complex entries, 246 KB) go
through the global buffer instead of shared memory.  Both solves are checked
by their normwise backward error against the library's own exported K, M, C
(the oracle's Python factorisation of this 103,041-DOF system would take
minutes); the same code paths at smaller sizes are oracle-checked in
test_gpu_parity.py and test_gpu_complex.py.
"""
import numpy as np
import pytest
import scipy.sparse as sp

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
