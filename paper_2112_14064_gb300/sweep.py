"""IGA against rIGA over mesh sizes: factorisation and FB cost on one GPU.

    python -m paper_2112_14064_gb300.sweep [--ne 256 512 1024 2048] [--p 3] [--block 16]
                                           [--solves 5] [--eigs-max-ne 1024]

For each ne the maximum-continuity IGA space (block 0) and the rIGA space
with C^0 lines every `block` elements are analysed and factorised at shift 0
in FP64; then `solves` FB solves are timed, and, up to --eigs-max-ne, the
in-region eigensolve of the 20 eigenpairs nearest 500 (shift 0, 56
candidates, Krylov dimension 96) runs on the factor.  One JSON line per
(ne, space) with the exact (elimination-tree) factor flops and entries, the
device times (CUDA events) and the rIGA/IGA ratios; this is the scalar H^1
analogue of the paper's Table 2 sweep.  Damping sigma_e ~ U[0.1, 1] per
element (seed 20211233).
"""
import argparse
import json
import statistics

import numpy as np


def run(ne, p, block, solves, eigs):
    import torch
    from paper_2112_14064_gb300 import rigaqep
    rng = np.random.default_rng(20211233)
    sig = torch.from_numpy(rng.uniform(0.1, 1.0, ne * ne)).cuda()
    pr = rigaqep.Problem(ne, p, block, sig).analyze()
    pr.factor(0.0)
    inf = pr.info()
    out = {"ne": ne, "p": p, "block": block, "space": "IGA" if block == 0 else "rIGA",
           "N": inf["N"], "nnz_L_exact": inf["nnz_L_exact"],
           "factor_flops_exact": inf["factor_flops_exact"], "nnz_L_stored": inf["nnz_L"],
           "factor_ms": inf["factor_ms"],
           "factor_tflops": inf["factor_flops_exact"] / (inf["factor_ms"] * 1e-3) / 1e12}
    b = torch.randn(inf["N"], dtype=torch.float64, device="cuda")
    x = torch.empty_like(b)
    pr.solve(b, out=x)
    ms = []
    for _ in range(solves):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        pr.solve(b, out=x)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    out["fb_ms_per_solve"] = statistics.median(ms)
    if eigs:
        lam, X, eta, nconv, st = pr.eigs(20, 500.0, m=96, shift=0.0, ncand=56, seed=1,
                                         raise_on_noconv=False)
        ie = pr.info()
        out.update(eigs_ms=ie["eigs_ms"], n_apply=ie["n_apply"], certified=ie["certified"],
                   converged=int(nconv), max_eta=float(eta.max().item()))
    pr.close()
    torch.cuda.synchronize()
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--ne", type=int, nargs="+", default=[256, 512, 1024, 2048])
    ap.add_argument("--p", type=int, default=3)
    ap.add_argument("--block", type=int, default=16)
    ap.add_argument("--solves", type=int, default=5)
    ap.add_argument("--eigs-max-ne", type=int, default=1024)
    a = ap.parse_args()
    for ne in a.ne:
        rows = {}
        for block in (0, a.block):
            rows[block] = run(ne, a.p, block, a.solves, ne <= a.eigs_max_ne)
            print(json.dumps(rows[block]), flush=True)
        iga, riga = rows[0], rows[a.block]
        ratio = {"ne": ne, "riga_over_iga": {
            "factor_flops": iga["factor_flops_exact"] / riga["factor_flops_exact"],
            "factor_entries": iga["nnz_L_exact"] / riga["nnz_L_exact"],
            "factor_time": iga["factor_ms"] / riga["factor_ms"],
            "fb_time": iga["fb_ms_per_solve"] / riga["fb_ms_per_solve"]}}
        if "eigs_ms" in iga and "eigs_ms" in riga:
            ratio["riga_over_iga"]["eigs_time"] = iga["eigs_ms"] / riga["eigs_ms"]
        print(json.dumps(ratio), flush=True)


if __name__ == "__main__":
    main()
