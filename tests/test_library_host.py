"""CPU-only checks of the C-ABI library: it loads, exports every declared
symbol, and its host symbolic phase is bit-exact against the oracle."""
import os
import re

import numpy as np
import pytest

from oracle import bspline
from oracle.assemble import assemble
from oracle.nd import symbolic
from paper_2112_14064_gb300 import rigaqep

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2112_14064_gb300 import build
    build.build()
    return rigaqep.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "rigaqep.h")).read()
    return sorted(set(re.findall(r"\b(rigaqep_[a-z_]+)\s*\(", src)))


def test_header_symbols_exported(lib):
    names = _declared()
    assert set(names) == set(rigaqep.EXPORTS)
    for n in names:
        assert hasattr(lib, n), n


def test_bad_mesh_is_rejected(lib):
    with pytest.raises(rigaqep.RigaqepError) as e:
        rigaqep.symbolic_host(16, 2, 5)          # block does not divide ne
    assert e.value.code == 1
    with pytest.raises(rigaqep.RigaqepError):
        rigaqep.symbolic_host(16, 1, 4)          # p < 2
    with pytest.raises(rigaqep.RigaqepError):
        rigaqep.symbolic_host(16, 9, 4)          # p > 8


def _oracle_sym(ne, p, b, rowptr=None, col=None):
    sp1 = bspline.Space1D(ne, p, b)
    if rowptr is None:
        A = assemble(ne, p, b, np.ones(ne * ne))
        rowptr, col = A.indptr, A.indices
    return symbolic(sp1.n, sp1.c0_dofs, p, rowptr, col, use_c0=b > 0)


@pytest.mark.parametrize("ne,p,b", [(16, 2, 4), (64, 3, 16), (10, 2, 0), (32, 5, 8),
                                    (16, 4, 8), (2, 2, 0), (3, 3, 0), (8, 2, 2)])
def test_host_symbolic_bit_exact(lib, ne, p, b):
    g = rigaqep.symbolic_host(ne, p, b)
    A = assemble(ne, p, b, np.ones(ne * ne))
    assert np.array_equal(g["rowptr"], A.indptr) and np.array_equal(g["col"], A.indices)
    s = _oracle_sym(ne, p, b, A.indptr, A.indices)
    for k in ("perm", "sptr", "parent", "upd_ptr", "upd_idx", "level"):
        assert np.array_equal(getattr(s, k), g[k]), k


@pytest.mark.slow
@pytest.mark.parametrize("ne,p,b", [(256, 3, 16), (256, 3, 0), (512, 3, 16)])
def test_host_symbolic_bit_exact_full_size(lib, ne, p, b):
    """Full-size workloads: the oracle runs on the library's pattern, which
    the small cases above pin against the oracle's own assembly."""
    g = rigaqep.symbolic_host(ne, p, b)
    s = _oracle_sym(ne, p, b, g["rowptr"].astype(np.int64), g["col"].astype(np.int64))
    for k in ("perm", "sptr", "parent", "upd_ptr", "upd_idx", "level"):
        assert np.array_equal(getattr(s, k), g[k]), k


@pytest.mark.parametrize("ne,p,b", [(16, 2, 4), (64, 3, 16), (10, 2, 0), (32, 5, 8), (24, 4, 0)])
def test_host_factor_counts_match_oracle(lib, ne, p, b):
    """Supernodal and exact nnz(L) / flop counts of the library's plan equal
    the oracle's (which tests/test_oracle_pins.py pins to brute-force
    elimination)."""
    g = rigaqep.symbolic_host(ne, p, b)
    A = assemble(ne, p, b, np.ones(ne * ne))
    s = _oracle_sym(ne, p, b, A.indptr, A.indices)
    assert g["nnz_L"] == s.nnz_L()
    assert g["factor_flops"] == s.factor_flops()
    assert g["nnz_L_exact"] == s.nnz_L_scalar(A.indptr, A.indices)
    assert g["factor_flops_exact"] == s.factor_flops_scalar(A.indptr, A.indices)


def test_host_exact_counts_full_size(lib):
    """256 x 256, p = 3, blocks of 16: the exact counts (7,291,970 entries,
    841,058,277 flops) are those of the oracle's elimination-tree count on the
    same plan; the supernodal ones are 8,669,570 and 1,067,962,341."""
    g = rigaqep.symbolic_host(256, 3, 16)
    assert (g["nnz_L_exact"], g["factor_flops_exact"]) == (7291970, 841058277)
    assert (g["nnz_L"], g["factor_flops"]) == (8669570, 1067962341)
