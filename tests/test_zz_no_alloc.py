"""The allocation-free damping gradient, through the C-ABI.

rigaqep_grad_damping_noalloc serves callers that must not allocate device
memory during the call (a latency-critical path that cannot afford the
device-wide synchronisation of cudaMalloc/cudaFree, or a framework whose own
memory manager owns the device).  It must give the same result as
rigaqep_grad_damping, also on a second call in a row (its scratch array keeps
the previous call's contents).  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2112_14064_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# the gradient tolerance of the parity tests (relative to the largest entry)
RTOL = 1e-8


@pytest.fixture(scope="module")
def rq():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_14064_gb300 import build, rigaqep
    build.build()
    rigaqep.load()
    return rigaqep


def test_noalloc_gradient_matches_allocating_entry_point(rq):
    c = dict(workloads.CONFIGS["tiny"])
    pr = rq.Problem(c["ne"], c["p"], c["block"], workloads.sigma_e(c)).analyze()
    lam, X, eta, nconv, st = pr.eigs(c["neig"], c["shift"], m=c["m"], seed=1)
    assert st == 0
    ref = pr.grad_damping(lam, X).cpu().numpy()
    scale = np.abs(ref).max()
    for call in range(2):   # the shared scratch keeps the previous call's contents
        out = torch.full((c["neig"], c["ne"] ** 2, 2), float("nan"), dtype=torch.float64,
                         device="cuda")
        G = pr.grad_damping_noalloc(lam, X, out=out).cpu().numpy()
        assert np.isfinite(G).all()
        assert np.abs(G - ref).max() <= RTOL * scale, call
    # a different, smaller request afterwards still reads only what it wrote
    G4 = pr.grad_damping_noalloc(lam[:4].contiguous(), X[:4].contiguous()).cpu().numpy()
    assert np.abs(G4 - ref[:4]).max() <= RTOL * scale
    pr.close()


def test_noalloc_gradient_rejects_too_many_pairs(rq):
    c = dict(workloads.CONFIGS["tiny"])
    pr = rq.Problem(c["ne"], c["p"], c["block"], workloads.sigma_e(c)).analyze()
    lib = rq.load()
    # real (small) device buffers: the size check comes first, but a wrong
    # order would then give a wrong status, never a stray device address
    buf = torch.zeros(64, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    code = lib.rigaqep_grad_damping_noalloc(pr._h, 65, p, p, p)
    assert code == 1
    assert b"64" in lib.rigaqep_last_error()
    pr.close()
