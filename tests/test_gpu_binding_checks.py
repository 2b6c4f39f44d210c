"""The Python binding rejects tensors the C-ABI would read or write past
their end (wrong dtype, shape, device or layout) before any library call:
the library takes plain device pointers and trusts the sizes it derives
from the problem."""
import numpy as np
import pytest

from paper_2112_14064_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def problem():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_14064_gb300 import build, rigaqep
    build.build()
    rigaqep.load()
    c = workloads.CONFIGS["tiny"]
    pr = rigaqep.Problem(c["ne"], c["p"], c["block"], workloads.sigma_e(c)).analyze().factor(20.0)
    yield pr
    pr.close()


def test_solve_checks_its_tensors(problem):
    pr = problem
    good = torch.ones(pr.N, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        pr.solve(good.float())                                  # float32 right-hand side
    with pytest.raises(ValueError):
        pr.solve(good[: pr.N - 1])                              # one entry short
    with pytest.raises(ValueError):
        pr.solve(good.cpu())                                    # host tensor
    with pytest.raises(ValueError):
        pr.solve(good, out=torch.empty(pr.N - 1, dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        pr.solve(good, out=torch.empty(pr.N, dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError):
        pr.solve(torch.ones((2, pr.N), dtype=torch.float64, device="cuda"),
                 out=torch.empty((pr.N, 2), dtype=torch.float64, device="cuda").t())
    x = pr.solve(good)                                          # the valid call still works
    assert x.shape == (pr.N,) and torch.isfinite(x).all()


def test_complex_solve_and_gradient_check_their_tensors(problem):
    pr = problem
    with pytest.raises(ValueError):
        pr.solve_complex(torch.ones(pr.N + 1, dtype=torch.complex128, device="cuda"))
    lam = torch.ones(3, dtype=torch.complex128, device="cuda")
    X = torch.ones((3, pr.N), dtype=torch.complex128, device="cuda")
    with pytest.raises(ValueError):
        pr.grad_damping(lam.to(torch.complex64), X)
    with pytest.raises(ValueError):
        pr.grad_damping(lam, X[:, 1:])
    with pytest.raises(ValueError):
        pr.grad_damping(lam[:2], X)
    with pytest.raises(ValueError):
        pr.grad_damping_noalloc(lam, X, out=torch.empty((3, 4, 2), dtype=torch.float64,
                                                         device="cuda"))


def test_start_vectors_are_checked(problem):
    pr = problem
    c = workloads.CONFIGS["tiny"]
    with pytest.raises(ValueError):
        pr.eigs(c["neig"], c["shift"], m=c["m"],
                v1=torch.ones(pr.N, dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        pr.eigs_undamped(1.0, 100.0, v1=torch.ones(2 * pr.N, dtype=torch.float64,
                                                   device="cuda"))
    rng = np.random.default_rng(3)
    v1 = torch.from_numpy(rng.standard_normal(2 * pr.N)).cuda()
    lam, X, eta, nconv, st = pr.eigs(c["neig"], c["shift"], m=c["m"], v1=v1,
                                     raise_on_noconv=False)
    assert nconv == c["neig"] and float(eta.max()) <= 1e-10
