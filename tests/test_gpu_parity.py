"""GPU parity: the CUDA path through the C-ABI against the FP64 CPU oracle.

Tolerances (FP64 everywhere):
* symbolic phase and CSR pattern: bit-exact;
* assembled values: 1e-13 relative to the largest entry (summation order of
  the element contributions differs);
* FB solve: 1e-11 relative (both are backward-stable solves of an SPD system
  whose condition number here is below 1e3);
* eigenvalues: 1e-10 relative, compared as multisets; backward errors eta
  <= 1e-10 (the target accuracy of the eigensolve);
* eigenvectors: through eta and the normalisation convention;
* gradients: 1e-8 relative to the largest entry (they inherit the
  eigenvector error, which for these separated eigenvalues is ~1e-11).
"""
import numpy as np
import pytest

from oracle.assemble import assemble
from oracle.multifrontal import factorize
from oracle.nd import symbolic
from oracle import qep
from oracle.adjoint import damping_gradient
from paper_2112_14064_gb300 import workloads
from eigmatch import multiset_max_rel, same_multiset

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


def _cfg(name, **over):
    c = dict(workloads.CONFIGS[name])
    c.update(over)
    return c


def _oracle(c):
    A = assemble(c["ne"], c["p"], c["block"], workloads.sigma_e(c))
    sym = symbolic(A.n1, A.space.c0_dofs, c["p"], A.indptr, A.indices, use_c0=c["block"] > 0)
    return A, sym


def _problem(rq, c):
    return rq.Problem(c["ne"], c["p"], c["block"], workloads.sigma_e(c)).analyze()



MESHES = [("tiny", {}), ("p3_64_b16", {}), ("tiny", dict(block=0)),
          ("tiny", dict(ne=8, p=5, block=8)), ("tiny", dict(ne=12, p=4, block=4)),
          ("tiny", dict(ne=2, p=2, block=0))]


@pytest.mark.parametrize("name,over", MESHES)
def test_assembly_and_symbolic(rq, name, over):
    c = _cfg(name, **over)
    A, sym = _oracle(c)
    pr = _problem(rq, c)
    csr = pr.export_csr()
    assert np.array_equal(csr["rowptr"], A.indptr) and np.array_equal(csr["col"], A.indices)
    for key, ref in (("K", A.K), ("M", A.M), ("C", A.C)):
        scale = np.abs(ref.data).max()
        assert np.abs(csr[key] - ref.data).max() <= 1e-13 * scale, key
    g = pr.export_symbolic()
    for k in ("perm", "sptr", "parent", "upd_ptr", "upd_idx", "level"):
        assert np.array_equal(getattr(sym, k), g[k]), k
    inf = pr.info()
    assert inf["nnz_L"] == sym.nnz_L() and inf["factor_flops"] == sym.factor_flops()
    assert inf["norm_K"] == pytest.approx(abs(A.K).sum(axis=1).max(), rel=1e-13)
    pr.close()


@pytest.mark.parametrize("name,over,sigma", [("tiny", {}, 20.0), ("p3_64_b16", {}, 800.0),
                                             ("tiny", dict(block=0), 5.0),
                                             ("tiny", dict(ne=8, p=5, block=8), 300.0)])
def test_solve_matches_oracle(rq, name, over, sigma):
    c = _cfg(name, **over)
    A, sym = _oracle(c)
    F = factorize(sym, A.Q(sigma))
    pr = _problem(rq, c).factor(sigma)
    rng = np.random.default_rng(7)
    B = rng.standard_normal((3, A.N))
    Xg = pr.solve(torch.from_numpy(B).cuda()).cpu().numpy()
    Xt = pr.solve(torch.from_numpy(B).cuda(), transpose=1).cpu().numpy()
    for i in range(3):
        ref = F.solve(B[i])
        assert np.abs(Xg[i] - ref).max() <= 1e-11 * np.abs(ref).max()
    assert np.array_equal(Xg, Xt)   # Q symmetric: the same path
    pr.close()


@pytest.mark.parametrize("ne,sigma,prec", [(128, 0.0, 0), (128, 500.0, 0), (256, 0.0, 0),
                                           (128, 0.0, 2)])
def test_solve_residual_large_fronts(rq, ne, sigma, prec):
    """Meshes whose top pivot blocks (143 and 287 pivots) are factorised by a
    cluster of CTAs: the FP64 residual of the GPU solve against the assembled
    Q(sigma) (a property that holds at any size; these systems have condition
    numbers below 1e7, so a backward-stable solve leaves < 1e-12)."""
    import scipy.sparse as sp
    c = _cfg("p3_256_b16", ne=ne)
    pr = _problem(rq, c).factor(sigma, prec)
    csr = pr.export_csr()
    Q = sp.csr_matrix((sigma * sigma * csr["M"] + sigma * csr["C"] + csr["K"], csr["col"],
                       csr["rowptr"]), shape=(pr.N, pr.N))
    B = np.random.default_rng(11).standard_normal((2, pr.N))
    X = pr.solve(torch.from_numpy(B).cuda()).cpu().numpy()
    for i in range(2):
        res = np.abs(B[i] - Q @ X[i]).max() / (np.abs(Q).max() * np.abs(X[i]).max())
        assert res <= 1e-12, res
    pr.close()


def test_solve_in_place_and_zero_rhs(rq):
    c = _cfg("tiny")
    A, _ = _oracle(c)
    pr = _problem(rq, c).factor(20.0)
    b = torch.from_numpy(np.random.default_rng(1).standard_normal(A.N)).cuda()
    x = pr.solve(b.clone())
    y = b.clone()
    pr.solve(y, out=y)                 # b and x alias
    assert torch.equal(x, y)
    empty = torch.empty((0, A.N), dtype=torch.float64, device="cuda")
    assert pr.solve(empty).shape == (0, A.N)
    pr.close()


EIGS = [("tiny", {}, None), ("tiny", dict(sigma_law="constant", value=0.4), None),
        ("tiny", dict(sigma_law="constant", value=0.0), None),
        ("p3_64_b16", dict(shift=20.0, neig=10, m=40), None),
        ("tiny", dict(block=0, shift=5.0, neig=6, m=24), None),
        ("tiny", dict(ne=8, p=5, block=8, shift=50.0, neig=4, m=16), None)]


@pytest.mark.parametrize("name,over,_", EIGS)
def test_eigs_match_oracle(rq, name, over, _):
    c = _cfg(name, **over)
    A, sym = _oracle(c)
    s, neig, m = c["shift"], c["neig"], c["m"]
    v1 = workloads.start_vector(1, 2 * A.N)
    F = factorize(sym, A.Q(s))
    ref = qep.eigs(A.K, A.C, A.M, s, neig, m, F.solve, v1)
    assert ref.n_conv == neig
    pr = _problem(rq, c)
    lam, X, eta, nconv, st = pr.eigs(neig, s, m=m, v1=torch.from_numpy(v1).cuda())
    lam = lam.cpu().numpy()
    X = X.cpu().numpy()
    eta = eta.cpu().numpy()
    assert nconv == neig and st == 0
    assert same_multiset(ref.lam, lam, 1e-10)
    assert eta.max() <= 1e-10
    # ordering: non-decreasing distance to the shift, Im > 0 first on ties
    d = np.abs(lam - s)
    assert np.all(np.diff(d) >= -1e-9 * d[:-1])
    # (only where the value is not repeated: repeated eigenvalues, e.g. the
    # symmetric modes of a constant-damping square, compare as multisets)
    def isolated(v):
        return np.sum(np.abs(lam - v) <= 1e-8 * abs(v)) == 1
    for k in range(neig - 1):
        if (abs(lam[k] - np.conj(lam[k + 1])) <= 1e-12 * abs(lam[k]) and lam[k].imag != 0
                and isolated(lam[k])):
            assert lam[k].imag > 0
    # the oracle's output order, value by value, for isolated values
    for k in range(neig):
        if isolated(lam[k]):
            assert abs(lam[k] - ref.lam[k]) <= 1e-10 * abs(ref.lam[k])
    for k in range(neig):
        x = X[k]
        assert np.linalg.norm(x) == pytest.approx(1.0, abs=1e-12)
        # an entry of largest modulus is real and positive; entries whose
        # moduli tie within rounding (symmetric modes) may each be the one
        ax = np.abs(x)
        top = np.flatnonzero(ax >= ax.max() * (1 - 1e-12))
        assert any(abs(x[i].imag) <= 1e-14 and x[i].real > 0 for i in top)
        # the oracle's own backward error of the GPU pair
        assert qep.backward_error(lam[k], x, A.K, A.C, A.M) <= 1e-10
    inf = pr.info()
    assert inf["n_apply"] >= m
    pr.close()


def test_eigs_device_start_vector_matches_generator(rq):
    """v1 = NULL: the device splitmix64 stream equals the input generator's."""
    c = _cfg("tiny")
    pr = _problem(rq, c)
    v1 = workloads.start_vector(1, 2 * pr.N)
    a = pr.eigs(c["neig"], c["shift"], m=c["m"], v1=torch.from_numpy(v1).cuda())
    b = pr.eigs(c["neig"], c["shift"], m=c["m"], seed=1)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    pr.close()


def test_gradient_matches_oracle(rq):
    c = _cfg("tiny")
    A, sym = _oracle(c)
    pr = _problem(rq, c)
    lam, X, eta, nconv, _ = pr.eigs(c["neig"], c["shift"], m=c["m"], seed=1)
    G = pr.grad_damping(lam, X).cpu().numpy()
    lam_h, X_h = lam.cpu().numpy(), X.cpu().numpy()
    ref = damping_gradient(c["ne"], c["p"], c["block"], lam_h, X_h, A.C, A.M)
    assert np.abs(G - ref).max() <= 1e-8 * np.abs(ref).max()
    pr.close()


@pytest.mark.parametrize("p,ne,block", [(2, 12, 0), (3, 12, 4), (4, 10, 5), (5, 8, 4),
                                         (6, 8, 4), (7, 8, 8)])
def test_gradient_every_degree(rq, p, ne, block):
    """Element gradients at each degree (register kernels for p = 2..5, the
    generic one otherwise) against the oracle's on the same eigenpairs."""
    c = _cfg("tiny", p=p, ne=ne, block=block, neig=6, m=30)
    A, _ = _oracle(c)
    pr = _problem(rq, c)
    lam, X, *_ = pr.eigs(c["neig"], c["shift"], m=c["m"], seed=1)
    G = pr.grad_damping(lam, X).cpu().numpy()
    ref = damping_gradient(c["ne"], c["p"], c["block"], lam.cpu().numpy(), X.cpu().numpy(),
                           A.C, A.M)
    assert np.abs(G - ref).max() <= 1e-10 * np.abs(ref).max()
    pr.close()


def test_gradient_sum_rule_constant_damping(rq):
    cst = 0.4
    c = _cfg("tiny", sigma_law="constant", value=cst)
    pr = _problem(rq, c)
    lam, X, *_ = pr.eigs(c["neig"], c["shift"], m=c["m"], seed=1)
    G = pr.grad_damping(lam, X).cpu().numpy()
    lam = lam.cpu().numpy()
    np.testing.assert_allclose(G.sum(axis=1), -lam / (2 * lam + cst), rtol=1e-9)
    pr.close()


def test_errors_are_reported(rq):
    c = _cfg("tiny")
    pr = rq.Problem(c["ne"], c["p"], c["block"], workloads.sigma_e(c))
    with pytest.raises(rq.RigaqepError) as e:
        pr.factor(20.0)                       # analyze has not run
    assert e.value.code == 2
    pr.analyze()
    with pytest.raises(rq.RigaqepError) as e:
        pr.solve(torch.zeros(pr.N, dtype=torch.float64, device="cuda"))
    assert e.value.code == 2
    with pytest.raises(rq.RigaqepError) as e:
        pr.eigs(10, -3.0)                      # shift must be > 0
    assert e.value.code == 1
    pr.close()
    # heavy damping makes Q(-1) = K - 99 M indefinite: reported, not trapped
    pr = rq.Problem(c["ne"], c["p"], c["block"], np.full(c["ne"] ** 2, 100.0)).analyze()
    with pytest.raises(rq.RigaqepError) as e:
        pr.factor(-1.0)
    assert e.value.code == 5
    pr.factor(20.0)                            # the handle stays usable
    pr.close()


def test_no_convergence_returns_partial(rq):
    c = _cfg("tiny")
    pr = _problem(rq, c)
    lam, X, eta, nconv, st = pr.eigs(c["neig"], c["shift"], m=c["m"], max_restarts=1,
                                     tol=1e-15, raise_on_noconv=False)
    assert st == 7 and nconv < c["neig"]
    pr.close()


@pytest.mark.slow
def test_full_size_p3_256_b16(rq):
    """The bench workload in the bench's launch configuration (256 x 256,
    p = 3, blocks of 16, target 500, 20 pairs; in-region shift 0 with 56
    candidates and m = 96): symbolic bit-exact, sampled assembled entries,
    solve residual, the certificate, the eigenvalues against the oracle's
    full solve of the same configuration (multiset, 1e-10 relative), and
    every returned pair checked with the oracle's own matrices (backward
    error <= 1e-10)."""
    import scipy.sparse as sp
    c = _cfg("p3_256_b16")
    sig = workloads.sigma_e(c)
    A = assemble(c["ne"], c["p"], c["block"], sig)
    pr = rq.Problem(c["ne"], c["p"], c["block"], sig).analyze()
    csr = pr.export_csr()
    assert np.array_equal(csr["rowptr"], A.indptr) and np.array_equal(csr["col"], A.indices)
    idx = np.random.default_rng(3).choice(A.K.nnz, 5000, replace=False)
    for key, ref in (("K", A.K), ("M", A.M), ("C", A.C)):
        assert np.abs(csr[key][idx] - ref.data[idx]).max() <= 1e-13 * np.abs(ref.data).max()
    sym = symbolic(A.n1, A.space.c0_dofs, c["p"], A.indptr, A.indices)
    g = pr.export_symbolic()
    for k in ("perm", "sptr", "parent", "upd_ptr", "upd_idx", "level"):
        assert np.array_equal(getattr(sym, k), g[k]), k
    s = c["shift"]
    pr.factor(s)
    Q = A.Q(s)
    b = np.random.default_rng(5).standard_normal(A.N)
    x = pr.solve(torch.from_numpy(b).cuda()).cpu().numpy()
    nQ = abs(Q).sum(axis=1).max()
    assert np.linalg.norm(Q @ x - b) <= 1e-13 * nQ * np.linalg.norm(x)
    v1 = workloads.start_vector(1, 2 * A.N)
    lam, X, eta, nconv, st = pr.eigs(c["neig"], s, m=96, v1=torch.from_numpy(v1).cuda(),
                                     shift=0.0, ncand=56)
    assert pr.info()["certified"] == 1
    lam, X, eta = lam.cpu().numpy(), X.cpu().numpy(), eta.cpu().numpy()
    assert nconv == c["neig"]
    F = factorize(sym, A.Q(0.0))
    ref = qep.eigs(A.K, A.C, A.M, 0.0, c["neig"], 96, F.solve, v1, target=s, ncand=56,
                   sigma_min=sig.min())
    assert ref.certified
    assert same_multiset(ref.lam, lam, 1e-10)
    for k in range(c["neig"]):
        assert qep.backward_error(lam[k], X[k], A.K, A.C, A.M) <= 1e-10
    assert eta.max() <= 1e-10
    pr.close()


@pytest.mark.parametrize("name,over,target,ncand,m", [
    ("tiny", {}, 20.0, 20, 40),
    ("p3_64_b16", {}, 500.0, 56, 72),
    ("tiny", dict(ne=12, p=4, block=4), 300.0, 40, 60)])
def test_in_region_shift_matches_oracle(rq, name, over, target, ncand, m):
    """Target/shift split: Q factorised at the in-region shift 0, ncand pairs
    converged there, the neig nearest the target returned and certified."""
    c = _cfg(name, **over)
    A, sym = _oracle(c)
    sig = workloads.sigma_e(c)
    v1 = workloads.start_vector(1, 2 * A.N)
    F = factorize(sym, A.Q(0.0))
    ref = qep.eigs(A.K, A.C, A.M, 0.0, c["neig"], m, F.solve, v1, target=target, ncand=ncand,
                   sigma_min=sig.min())
    assert ref.certified
    pr = _problem(rq, c)
    lam, X, eta, nconv, st = pr.eigs(c["neig"], target, m=m, v1=torch.from_numpy(v1).cuda(),
                                     shift=0.0, ncand=ncand)
    inf = pr.info()
    assert st == 0 and nconv == c["neig"] and inf["certified"] == 1
    lam = lam.cpu().numpy()
    assert same_multiset(ref.lam, lam, 1e-10)
    assert eta.max().item() <= 1e-10
    d = np.abs(lam - target)
    assert np.all(np.diff(d) >= -1e-9 * d[:-1])
    pr.close()


def test_in_region_agrees_with_literal_shift(rq):
    """Where the literal shift converges (tiny mesh, target 20) both modes
    return the same eigenvalues."""
    c = _cfg("tiny")
    pr = _problem(rq, c)
    a = pr.eigs(c["neig"], c["shift"], m=c["m"], seed=1)[0].cpu().numpy()
    b = pr.eigs(c["neig"], c["shift"], m=c["m"], seed=1, shift=0.0, ncand=20)[0].cpu().numpy()
    assert pr.info()["certified"] == 1
    assert same_multiset(a, b, 1e-10)
    pr.close()


@pytest.mark.parametrize("name,over,target,kw", [
    ("tiny", {}, 20.0, dict(m=40)),
    ("p3_64_b16", {}, 500.0, dict(m=72, shift=0.0, ncand=56))])
def test_scaled_pencil_matches_oracle(rq, name, over, target, kw):
    """Remark 4's scaled pencil (scaling=True) against the oracle's scaled
    solve: the same scaling factor, eigenvalues 1e-10 (multiset), eta <= 1e-10."""
    c = _cfg(name, **over)
    A, sym = _oracle(c)
    sig = workloads.sigma_e(c)
    v1 = workloads.start_vector(1, 2 * A.N)
    shift = kw.get("shift", target)
    F = factorize(sym, A.Q(shift))
    extra = dict(target=target, ncand=kw["ncand"], sigma_min=sig.min()) if "ncand" in kw else {}
    ref = qep.eigs_scaled(A.K, A.C, A.M, shift, c["neig"], kw["m"], F.solve, v1, **extra)
    pr = _problem(rq, c)
    lam, X, eta, nconv, st = pr.eigs(c["neig"], target, v1=torch.from_numpy(v1).cuda(),
                                     scaling=True, **kw)
    inf = pr.info()
    assert st == 0 and nconv == c["neig"]
    assert inf["scale_factor"] == pytest.approx(ref.scale, rel=1e-14)
    assert inf["certified"] == int(ref.certified)
    assert same_multiset(ref.lam, lam.cpu().numpy(), 1e-10)
    assert eta.max().item() <= 1e-10
    pr.close()


def test_scaled_pencil_full_size(rq):
    """256 x 256 bench workload: scaled and unscaled solves agree to 1e-10."""
    c = _cfg("p3_256_b16")
    kw = dict(m=96, shift=0.0, ncand=56, seed=1)
    pr = _problem(rq, c)
    a = pr.eigs(c["neig"], c["shift"], **kw)[0].cpu().numpy()
    lam, X, eta, nconv, st = pr.eigs(c["neig"], c["shift"], scaling=True, **kw)
    inf = pr.info()
    assert st == 0 and inf["certified"] == 1 and inf["scale_factor"] > 1.0
    assert same_multiset(a, lam.cpu().numpy(), 1e-10)
    assert eta.max().item() <= 1e-10
    pr.close()
