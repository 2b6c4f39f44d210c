"""Undamped pencil K x = mu M x on the GPU: inertia counts (spectrum slicing,
Section 4.1.4) and shift-and-invert Lanczos on a slice (Remark 3).

* Counts: the negative pivots of the GPU's LDL^T of K - mu M against
  LAPACK's symmetric-definite eigenvalues (tiny mesh) and against the
  oracle's own LDL^T (64 x 64, p = 3), exact.
* Slices: eigenvalues against the oracle's Lanczos slice (multiset, 1e-10),
  the count, the certificate, residuals <= 1e-10, and the two eigenvectors
  of each double eigenvalue (the square's x <-> y symmetry) independent.
* 256 x 256, p = 3: every eigenvalue in [500, 1000) against the Dirichlet
  Laplacian's pi^2 (m^2 + n^2) (the B-spline discretisation error at this
  resolution is below 1e-6 relative; the gaps between distinct values are
  far larger), and the count equals the number of those values.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle.assemble import assemble
from oracle.nd import symbolic
from oracle import gep
from paper_2112_14064_gb300 import workloads
from eigmatch import multiset_max_rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_14064_gb300 import build, rigaqep
    build.build()
    rigaqep.load()
    return rigaqep


def test_inertia_against_dense(rq):
    c = dict(workloads.CONFIGS["tiny"])
    sig = workloads.sigma_e(c)            # the damping is ignored by the undamped pencil
    A = assemble(c["ne"], c["p"], c["block"], sig)
    mu_all = sla.eigh(A.K.toarray(), A.M.toarray(), eigvals_only=True)
    pr = rq.Problem(c["ne"], c["p"], c["block"], sig).analyze()
    for mu in (1.0, 30.0, 123.4, 700.0, 5000.0, 1e5):
        assert pr.inertia(mu) == int((mu_all < mu).sum()), mu
    pr.close()


def test_inertia_against_oracle_64(rq):
    c = dict(workloads.CONFIGS["p3_64_b16"])
    sig = workloads.sigma_e(c)
    A = assemble(c["ne"], c["p"], c["block"], sig)
    sym = symbolic(A.n1, A.space.c0_dofs, c["p"], A.indptr, A.indices)
    pr = rq.Problem(c["ne"], c["p"], c["block"], sig).analyze()
    for mu in (200.0, 2000.0, 20000.0):
        assert pr.inertia(mu) == gep.inertia(sym, A.K, A.M, mu), mu
    pr.close()


@pytest.mark.parametrize("name,lo,hi", [("tiny", 100.0, 400.0), ("p3_64_b16", 500.0, 1000.0)])
def test_slice_against_oracle(rq, name, lo, hi):
    c = dict(workloads.CONFIGS[name])
    sig = workloads.sigma_e(c)
    A = assemble(c["ne"], c["p"], c["block"], sig)
    sym = symbolic(A.n1, A.space.c0_dofs, c["p"], A.indptr, A.indices)
    v1 = workloads.start_vector(1, 2 * A.N)[A.N:]
    ref_mu, ref_X, ref_count, ref_cert = gep.slice(sym, A.K, A.M, lo, hi, 96, v1)
    assert ref_cert
    pr = rq.Problem(c["ne"], c["p"], c["block"], sig).analyze()
    mu, X, res, count, cert = pr.eigs_undamped(lo, hi, seed=1)
    assert count == ref_count and cert == 1 and len(mu) == count
    mu = mu.cpu().numpy()
    X = X.cpu().numpy()
    assert multiset_max_rel(ref_mu, mu) < 1e-10
    assert np.all(np.diff(mu) >= 0)
    assert res.max().item() <= 1e-10
    for x, m_ in zip(X, mu):
        assert np.linalg.norm(x) == pytest.approx(1.0, abs=1e-12)
        assert gep.residual(A.K, A.M, m_, x) <= 1e-10
    # double eigenvalues: their two vectors span the 2-D eigenspace
    for i in range(len(mu) - 1):
        if abs(mu[i + 1] - mu[i]) <= 1e-8 * mu[i]:
            a, b = X[i], X[i + 1]
            cosang = abs(a @ (A.M @ b)) / np.sqrt((a @ (A.M @ a)) * (b @ (A.M @ b)))
            assert cosang < 0.99
    pr.close()


def test_slice_full_size_against_laplacian(rq):
    c = dict(workloads.CONFIGS["p3_256_b16"])
    pr = rq.Problem(c["ne"], c["p"], c["block"], workloads.sigma_e(c)).analyze()
    lo, hi = 500.0, 1000.0
    mu, X, res, count, cert = pr.eigs_undamped(lo, hi, seed=1)
    exact = np.array(sorted(np.pi ** 2 * (m * m + n * n) for m in range(1, 20)
                            for n in range(1, 20)))
    exact = exact[(exact >= lo) & (exact < hi)]
    assert count == len(exact) and cert == 1 and len(mu) == count
    assert multiset_max_rel(exact, mu.cpu().numpy()) < 1e-6
    assert res.max().item() <= 1e-10
    pr.close()


def test_undamped_arguments(rq):
    c = dict(workloads.CONFIGS["tiny"])
    pr = rq.Problem(c["ne"], c["p"], c["block"], workloads.sigma_e(c)).analyze()
    with pytest.raises(rq.RigaqepError) as e:
        pr.eigs_undamped(400.0, 100.0)          # empty interval
    assert e.value.code == 1
    with pytest.raises(rq.RigaqepError) as e:
        pr.eigs_undamped(10.0, 400.0, nmax=3)   # more eigenvalues than room
    assert e.value.code == 1
    mu, X, res, count, cert = pr.eigs_undamped(1.0, 10.0)   # none there
    assert count == 0 and cert == 1 and len(mu) == 0
    # the QEP solve still works after the undamped factorisations
    lam, X, eta, nconv, st = pr.eigs(c["neig"], c["shift"], m=c["m"], seed=1)
    assert st == 0 and nconv == c["neig"]
    pr.close()
