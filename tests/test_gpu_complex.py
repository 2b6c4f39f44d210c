"""Complex shift s (Section 4.1.1) on the GPU against the oracle.

* The complex symmetric LDL^T of Q(s) and its solves: 1e-11 relative to the
  oracle's complex solve (the shifted systems here are well conditioned).
* Eigenpairs nearest s from the real-operator Krylov-Schur with the
  quadratic back-mapping: 1e-10 relative (multiset) to the oracle's
  complex-shift solve on the same inputs, eta <= 1e-10.
* The mu-plane reading of the workloads (s = i sqrt(sigma)): the 256^2 mesh
  at s = i sqrt(500) and the p = 4, 512^2 lognormal-damping mesh at
  s = i sqrt(2000): every pair with eta <= 1e-10, ordered by |lambda - s|.
"""
import numpy as np
import pytest

from oracle.assemble import assemble
from oracle.multifrontal import factorize
from oracle.nd import symbolic
from oracle import qep
from paper_2112_14064_gb300 import workloads
from eigmatch import same_multiset

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


def _setup(name, shift):
    c = dict(workloads.CONFIGS[name])
    sig = workloads.sigma_e(c)
    A = assemble(c["ne"], c["p"], c["block"], sig)
    sym = symbolic(A.n1, A.space.c0_dofs, c["p"], A.indptr, A.indices)
    Q = (A.K + shift * A.C + shift * shift * A.M).tocsr()
    return c, sig, A, factorize(sym, Q)


@pytest.mark.parametrize("name,shift", [("tiny", 1j * np.sqrt(300.0)),
                                        ("p3_64_b16", 0.3 + 1j * np.sqrt(800.0))])
def test_complex_solve_matches_oracle(rq, name, shift):
    c, sig, A, F = _setup(name, shift)
    rng = np.random.default_rng(4)
    b = rng.standard_normal(A.N) + 1j * rng.standard_normal(A.N)
    ref = F.solve(b)
    pr = rq.Problem(c["ne"], c["p"], c["block"], sig).analyze().factor_complex(shift)
    x = pr.solve_complex(torch.from_numpy(b).cuda()).cpu().numpy()
    assert np.abs(x - ref).max() <= 1e-11 * np.abs(ref).max()
    pr.close()


@pytest.mark.parametrize("name,shift,neig,m", [("tiny", 1j * np.sqrt(300.0), 10, 40),
                                               ("p3_64_b16", 1j * np.sqrt(800.0), 20, 72)])
def test_complex_shift_eigs_match_oracle(rq, name, shift, neig, m):
    c, sig, A, F = _setup(name, shift)
    v1 = workloads.start_vector(1, 2 * A.N)
    ref = qep.eigs_complex_shift(A.K, A.C, A.M, shift, neig, m, F.solve, v1)
    pr = rq.Problem(c["ne"], c["p"], c["block"], sig).analyze()
    lam, X, eta, nconv, st = pr.eigs(neig, 1.0, m=m, shift=shift, v1=torch.from_numpy(v1).cuda())
    assert st == 0 and nconv == neig
    lam = lam.cpu().numpy()
    assert same_multiset(ref.lam, lam, 1e-10)
    assert eta.max().item() <= 1e-10
    d = np.abs(lam - shift)
    assert np.all(np.diff(d) >= -1e-9 * d[:-1])
    X = X.cpu().numpy()
    for k in range(neig):
        assert qep.backward_error(lam[k], X[k], A.K, A.C, A.M) <= 1e-10
    pr.close()


@pytest.mark.parametrize("name,sigma", [("p3_256_b16", 500.0), ("p4_512_b32", 2000.0)])
def test_complex_shift_workloads(rq, name, sigma):
    c = dict(workloads.CONFIGS[name])
    shift = 1j * np.sqrt(sigma)
    pr = rq.Problem(c["ne"], c["p"], c["block"],
                    torch.from_numpy(workloads.sigma_e(c)).cuda()).analyze()
    lam, X, eta, nconv, st = pr.eigs(20, 1.0, m=96, shift=shift, seed=1)
    assert st == 0 and nconv == 20
    assert eta.max().item() <= 1e-10
    lam = lam.cpu().numpy()
    d = np.abs(lam - shift)
    assert np.all(np.diff(d) >= -1e-9 * d[:-1])
    # the modes nearest i sqrt(sigma) oscillate near that frequency
    assert np.all(np.abs(lam.imag - np.sqrt(sigma)) < 0.25 * np.sqrt(sigma))
    pr.close()
