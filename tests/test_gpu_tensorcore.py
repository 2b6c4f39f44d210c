"""The tensor-core (tcgen05) product of the front factorisation on its own.

rigaqep_front_gemm runs C = A B^T through the same operand staging (each
FP32 operand split into two TF32 or BF16 terms) and the same tcgen05 / TMA
kernel as the RIGAQEP_TF32_IR / RIGAQEP_BF16_IR fronts.  Reference: the
FP64 product of the same FP32 inputs.  Bound: |C - C64| <= tol * (|A| |B|^T)
elementwise, with tol from the arithmetic of the split.

* TF32 terms keep 11 significant bits each, so x = hi + lo holds x to about
  2^-22 relative; the dropped lo*lo term is below 2^-22 of |a b|, and the FP32
  accumulation adds k 2^-24: tol = 4e-6 for the k used here (<= 300).
* BF16 terms keep 8 bits, x = hi + lo to 2^-16 (and lo*lo to 2^-16): tol =
  6e-5.

The sizes cover one tile, ragged tails in every dimension (m, n not
multiples of 128, k not a multiple of the 32 / 64-element K-block) and
several K-blocks per tile, beyond the three-stage ring.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"TF32_IR": 4e-6, "BF16_IR": 6e-5}
SIZES = [(1, 1, 1), (128, 128, 32), (200, 130, 49), (300, 257, 143), (129, 65, 300),
         (17, 300, 70)]


@pytest.fixture(scope="module")
def rq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_14064_gb300 import build, rigaqep
    build.build()
    rigaqep.load()
    return rigaqep


@pytest.mark.parametrize("prec", ["TF32_IR", "BF16_IR"])
@pytest.mark.parametrize("m,n,k", SIZES)
def test_front_gemm_against_fp64(rq, prec, m, n, k):
    g = np.random.default_rng(m * 1000 + n * 10 + k)
    # entries spanning a few orders of magnitude, as in the fronts
    A = (g.standard_normal((m, k)) * np.exp(g.uniform(-3, 3, (m, k)))).astype(np.float32)
    B = (g.standard_normal((n, k)) * np.exp(g.uniform(-3, 3, (n, k)))).astype(np.float32)
    C = rq.front_gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(),
                      precision=getattr(rq, prec)).cpu().numpy().astype(np.float64)
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    ref = A64 @ B64.T
    scale = np.abs(A64) @ np.abs(B64).T
    ratio = np.abs(C - ref) / scale
    assert np.all(np.isfinite(C))
    assert ratio.max() <= TOL[prec], ratio.max()


def test_front_gemm_two_terms_beat_one(rq):
    """The split is in effect: the TF32 result is far more accurate than a
    single TF32 rounding of the operands would allow (2^-11 relative)."""
    g = np.random.default_rng(7)
    A = g.standard_normal((256, 96)).astype(np.float32)
    B = g.standard_normal((192, 96)).astype(np.float32)
    C = rq.front_gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(),
                      precision=rq.TF32_IR).cpu().numpy().astype(np.float64)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    scale = np.abs(A.astype(np.float64)) @ np.abs(B.astype(np.float64)).T
    assert (np.abs(C - ref) / scale).max() < 2.0 ** -18


def test_front_gemm_arguments(rq):
    lib = rq.load()
    z = torch.zeros(4, dtype=torch.float32, device="cuda")
    p = z.data_ptr()
    # unsupported precision, bad sizes: rejected before any GPU work
    assert lib.rigaqep_front_gemm(rq.FP64, 1, 1, 1, p, p, p, None) == 1
    assert lib.rigaqep_front_gemm(rq.TF32_IR, 1, 1, 0, p, p, p, None) == 1
    assert lib.rigaqep_front_gemm(rq.TF32_IR, -1, 1, 1, p, p, p, None) == 1
    # empty product: nothing to do
    assert lib.rigaqep_front_gemm(rq.TF32_IR, 0, 4, 4, None, None, None, None) == 0
