"""Mixed precision on the GPU: FP32 factor storage and FP32 sweeps, every
solve refined in FP64 against the assembled K, M, C.  Three front
precisions: FP32 SIMT (RIGAQEP_FP32_IR), and the front products on the
tensor cores in split TF32 (RIGAQEP_TF32_IR) or split BF16
(RIGAQEP_BF16_IR).

Tolerances:
* solves: 1e-12 relative to the FP64 oracle solve (the refinement runs until
  the probe residual reaches 1e-14 or stops halving, and these Q(0) = K
  systems have condition numbers well below 1e6);
* eigenvalues: 1e-9 relative to the FP64 oracle (the mixed-mode accuracy the
  method is held to), backward errors eta <= 1e-10;
* at full size (256 x 256), the mixed eigenvalues against the FP64 GPU path:
  1e-9 relative.
"""
import numpy as np
import pytest

from oracle.assemble import assemble
from oracle.multifrontal import factorize
from oracle.nd import symbolic
from oracle import qep
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


def _oracle(c):
    A = assemble(c["ne"], c["p"], c["block"], workloads.sigma_e(c))
    sym = symbolic(A.n1, A.space.c0_dofs, c["p"], A.indptr, A.indices, use_c0=c["block"] > 0)
    return A, sym



PRECS = ["FP32_IR", "TF32_IR", "BF16_IR"]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name,sigma,over", [
    ("tiny", 0.0, {}), ("tiny", 20.0, {}), ("p3_64_b16", 0.0, {}),
    # fronts of several 128-row tiles and K-blocks: pivot blocks of 143 and
    # update blocks of up to 287 rows
    ("tiny", 5.0, dict(ne=128, p=3, block=16)),
    # degree 5: wide macroelement separators (k not a multiple of 32)
    ("tiny", 1.0, dict(ne=24, p=5, block=8))])
def test_mixed_solve_matches_oracle(rq, name, sigma, over, prec):
    c = dict(workloads.CONFIGS[name])
    c.update(over)
    A, sym = _oracle(c)
    F = factorize(sym, A.Q(sigma))
    b = np.random.default_rng(5).standard_normal((2, A.N))
    ref = np.stack([F.solve(bb) for bb in b])
    pr = rq.Problem(c["ne"], c["p"], c["block"], workloads.sigma_e(c)).analyze()
    pr.factor(sigma, getattr(rq, prec))
    inf = pr.info()
    assert inf["n_ir"] >= 1 and inf["ir_residual"] <= 1e-13
    x = pr.solve(torch.from_numpy(b).cuda()).cpu().numpy()
    err = np.abs(x - ref).max() / np.abs(ref).max()
    assert err <= 1e-12, err
    pr.close()


@pytest.mark.parametrize("prec", PRECS)
def test_mixed_eigs_literal_shift_matches_oracle(rq, prec):
    c = dict(workloads.CONFIGS["tiny"])
    A, sym = _oracle(c)
    v1 = workloads.start_vector(1, 2 * A.N)
    F = factorize(sym, A.Q(c["shift"]))
    ref = qep.eigs(A.K, A.C, A.M, c["shift"], c["neig"], c["m"], F.solve, v1)
    pr = rq.Problem(c["ne"], c["p"], c["block"], workloads.sigma_e(c)).analyze()
    lam, X, eta, nconv, st = pr.eigs(c["neig"], c["shift"], m=c["m"],
                                     v1=torch.from_numpy(v1).cuda(), precision=getattr(rq, prec))
    assert st == 0 and nconv == c["neig"]
    lam = lam.cpu().numpy()
    assert same_multiset(ref.lam, lam, 1e-9)
    assert eta.max().item() <= 1e-10
    pr.close()


@pytest.mark.parametrize("prec", PRECS)
def test_mixed_eigs_in_region_matches_oracle(rq, prec):
    c = dict(workloads.CONFIGS["p3_64_b16"])
    A, sym = _oracle(c)
    sig = workloads.sigma_e(c)
    v1 = workloads.start_vector(1, 2 * A.N)
    F = factorize(sym, A.Q(0.0))
    ref = qep.eigs(A.K, A.C, A.M, 0.0, c["neig"], 96, F.solve, v1, target=500.0, ncand=56,
                   sigma_min=sig.min())
    assert ref.certified
    pr = rq.Problem(c["ne"], c["p"], c["block"], sig).analyze()
    lam, X, eta, nconv, st = pr.eigs(c["neig"], 500.0, m=96, v1=torch.from_numpy(v1).cuda(),
                                     shift=0.0, ncand=56, precision=getattr(rq, prec))
    assert st == 0 and pr.info()["certified"] == 1
    lam = lam.cpu().numpy()
    assert same_multiset(ref.lam, lam, 1e-9)
    assert eta.max().item() <= 1e-10
    pr.close()


@pytest.mark.parametrize("prec", PRECS)
def test_mixed_against_fp64_full_size(rq, prec):
    """256 x 256, p = 3, blocks of 16, target 500 (the bench workload)."""
    c = dict(workloads.CONFIGS["p3_256_b16"])
    sig = torch.from_numpy(workloads.sigma_e(c)).cuda()
    kw = dict(m=96, shift=0.0, ncand=56, seed=1)
    pr = rq.Problem(c["ne"], c["p"], c["block"], sig).analyze()
    a = pr.eigs(c["neig"], c["shift"], **kw)[0].cpu().numpy()
    lam, X, eta, nconv, st = pr.eigs(c["neig"], c["shift"], precision=getattr(rq, prec), **kw)
    inf = pr.info()
    assert st == 0 and inf["certified"] == 1 and inf["n_ir"] >= 1
    b = lam.cpu().numpy()
    assert same_multiset(a, b, 1e-9)
    assert eta.max().item() <= 1e-10
    pr.close()


@pytest.mark.parametrize("prec", ["TF32_IR", "BF16_IR"])
def test_tile_autotuner_choice_is_reused(rq, prec):
    """The first tensor-core factorisation of a mesh times both tile widths
    of the L21 product per level and keeps the faster; a second handle of the
    same mesh reuses the choice, and both factors give the same solves."""
    c = dict(workloads.CONFIGS["p3_64_b16"])
    sig = workloads.sigma_e(c)
    out = []
    for _ in range(2):
        pr = rq.Problem(c["ne"], c["p"], c["block"], sig).analyze()
        b = torch.from_numpy(np.random.default_rng(9).standard_normal(pr.N)).cuda()
        pr.factor(0.0, getattr(rq, prec))
        inf = pr.info()
        assert inf["tc_wide_levels"] >= 0
        out.append((inf["tc_wide_levels"], pr.solve(b).cpu().numpy()))
        pr.close()
    assert out[0][0] == out[1][0]
    assert np.abs(out[0][1] - out[1][1]).max() <= 1e-12 * np.abs(out[0][1]).max()
