"""Batched eigensolves on the GPU: many independent QEPs of uneven size, each
with several targets, in one rigaqep_batch_eigs call.

* Every job returns exactly (bit for bit) what the single-problem path
  returns for the same handle inputs: the batch only schedules the same
  kernels on per-handle streams from host worker threads, and every device
  reduction has a fixed order.
* In-region jobs of one handle after the first reuse its converged
  candidates; a fresh solve with the later target gives the same result.
* A small batch problem matches the FP64 oracle (eigenvalues 1e-10 relative,
  backward errors <= 1e-10, selection certified).
* A failing job reports its own status without stopping the others.
"""
import numpy as np
import pytest

from oracle.assemble import assemble
from oracle.multifrontal import factorize
from oracle.nd import symbolic
from oracle import qep
from paper_2112_14064_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# ne, p, block of an uneven mix (the batch workload draws from the same ranges)
MIX = [(32, 2, 8), (16, 2, 4), (24, 3, 8), (16, 4, 4), (32, 3, 16), (40, 5, 8)]
REGION = dict(shift=0.0, ncand=32, m=64)


@pytest.fixture(scope="module")
def rq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_14064_gb300 import build, rigaqep
    build.build()
    rigaqep.load()
    return rigaqep


def _sig(ne, seed):
    return workloads.sigma_e(dict(ne=ne, sigma_law="uniform", lo=0.05, hi=2.0, seed=seed))


def _jobs():
    jobs = []
    for i in range(len(MIX)):
        for t in (15.0, 60.0):
            jobs.append(dict(problem=i, neig=6, target=t, seed=3 + i, **REGION))
    # a literal-shift job (the shift at the target) on the smallest problem
    jobs.append(dict(problem=1, neig=6, target=20.0, seed=1, m=30))
    return jobs


def _single(rq, i, job):
    ne, p, b = MIX[i]
    pr = rq.Problem(ne, p, b, _sig(ne, 100 + i)).analyze()
    kw = {k: job[k] for k in ("m", "seed", "shift", "ncand") if k in job}
    lam, X, eta, nconv, st = pr.eigs(job["neig"], job["target"], **kw)
    inf = pr.info()
    pr.close()
    return lam, X, eta, nconv, st, inf


def test_batch_matches_single_problem_path(rq):
    streams = [torch.cuda.Stream() for _ in MIX]
    probs = [rq.Problem(ne, p, b, _sig(ne, 100 + i), stream=streams[i])
             for i, (ne, p, b) in enumerate(MIX)]
    jobs = _jobs()
    res = rq.batch_eigs(probs, jobs, nthreads=4)
    torch.cuda.synchronize()
    for j, (job, r) in enumerate(zip(jobs, res)):
        assert r["status"] == 0, j
        lam, X, eta, nconv, st, inf = _single(rq, job["problem"], job)
        assert st == 0 and nconv == r["n_converged"] == job["neig"]
        assert torch.equal(lam, r["lam"]), j
        assert torch.equal(X, r["X"]), j
        assert torch.equal(eta, r["eta"]), j
        assert r["certified"] == inf["certified"]
        assert r["eta"].max().item() <= 1e-10
    # the second in-region target of every problem reused the candidates
    for j, job in enumerate(jobs):
        first = j == 0 or jobs[j - 1]["problem"] != job["problem"] or "shift" not in job
        assert res[j]["reused_candidates"] == (0 if first else 1), j
    for pr in probs:
        pr.close()


def test_reuse_equals_fresh_solve(rq):
    """Consecutive in-region calls on one handle: the reused selection for a
    second target is the one a fresh handle computes."""
    ne, p, b = MIX[2]
    pr = rq.Problem(ne, p, b, _sig(ne, 102)).analyze()
    pr.eigs(6, 15.0, seed=5, **REGION)
    lam, X, eta, *_ = pr.eigs(8, 60.0, seed=5, **REGION)
    assert pr.info()["reused_candidates"] == 1
    pr.close()
    fresh = rq.Problem(ne, p, b, _sig(ne, 102)).analyze()
    lam2, X2, eta2, *_ = fresh.eigs(8, 60.0, seed=5, **REGION)
    assert fresh.info()["reused_candidates"] == 0
    fresh.close()
    assert torch.equal(lam, lam2) and torch.equal(X, X2) and torch.equal(eta, eta2)


def test_batch_problem_matches_oracle(rq):
    i = 3
    ne, p, b = MIX[i]
    sig = _sig(ne, 100 + i)
    A = assemble(ne, p, b, sig)
    sym = symbolic(A.n1, A.space.c0_dofs, p, A.indptr, A.indices, use_c0=b > 0)
    F = factorize(sym, A.Q(0.0))
    v1 = workloads.start_vector(3 + i, 2 * A.N)
    probs = [rq.Problem(ne, p, b, sig, stream=torch.cuda.Stream())]
    jobs = [dict(problem=0, neig=6, target=t, seed=3 + i, **REGION) for t in (15.0, 60.0)]
    res = rq.batch_eigs(probs, jobs)
    for job, r in zip(jobs, res):
        ref = qep.eigs(A.K, A.C, A.M, 0.0, 6, REGION["m"], F.solve, v1, target=job["target"],
                       ncand=REGION["ncand"], sigma_min=sig.min())
        assert ref.certified and r["certified"] == 1
        lam = r["lam"].cpu().numpy()
        err = max(np.min(np.abs(ref.lam - g)) / abs(g) for g in lam)
        err2 = max(np.min(np.abs(lam - g)) / abs(g) for g in ref.lam)
        assert err < 1e-10 and err2 < 1e-10
        assert r["eta"].max().item() <= 1e-10
    probs[0].close()


def test_failing_job_does_not_stop_the_batch(rq):
    probs = [rq.Problem(ne, p, b, _sig(ne, 100 + i), stream=torch.cuda.Stream())
             for i, (ne, p, b) in enumerate(MIX[:2])]
    jobs = [dict(problem=0, neig=6, target=15.0, seed=1, **REGION),
            dict(problem=1, neig=40, target=15.0, seed=1, **REGION),   # neig > ncand
            dict(problem=1, neig=6, target=15.0, seed=1, **REGION)]
    res = rq.batch_eigs(probs, jobs, raise_on_error=False)
    assert [r["status"] for r in res] == [0, 1, 0]
    with pytest.raises(rq.RigaqepError) as ei:
        rq.batch_eigs(probs, jobs)
    assert "batch job 1" in str(ei.value)
    for pr in probs:
        pr.close()
