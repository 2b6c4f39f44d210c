"""Per-stage timing of the rIGA QEP path on one synthetic workload.

    python -m paper_2112_14064_gb300.stages --workload p3_256_b16 --stage solve --reps 5

runs the path up to the chosen stage once, then repeats that stage ``reps``
times and prints one JSON line with the CUDA-event time of every repetition
(on the library's stream).  Stages:

* ``assemble`` - Problem(): CSR pattern on the host, Gauss-quadrature K, M, C
  on the device;
* ``analyze``  - nested dissection, supernodal symbolic phase, front maps;
* ``factor``   - multifrontal LDL^T of Q(shift);
* ``solve``    - one forward/backward solve with the factor (one right-hand
  side, seeded);
* ``eigs``     - the shift-and-invert Krylov-Schur eigensolve with the
  workload's target, in-region shift and candidate count.

It is also the program that the kernel-level profiles are captured on: a
small ``--reps`` keeps a profiler capture short.
"""
import argparse
import json
import time

import torch

from . import rigaqep, workloads

# in-region eigensolve options of each workload: (Krylov dimension, shift, candidates)
EIGS_OPTS = {
    "p3_256_b16": dict(m=96, shift=0.0, ncand=56),
    "p3_64_b16": dict(m=96, shift=0.0, ncand=80),
    "p3_256_iga": dict(m=96, shift=0.0, ncand=56),
}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--workload", default="p3_256_b16", choices=sorted(workloads.CONFIGS))
    ap.add_argument("--stage", default="solve",
                    choices=["assemble", "analyze", "factor", "solve", "eigs"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--factor-shift", type=float, default=0.0)
    ap.add_argument("--precision", default="FP64", choices=["FP64", "TF32_IR", "FP32_IR", "BF16_IR"],
                    help="front precision of the factor, solve and eigs stages")
    a = ap.parse_args(argv)
    if a.reps < 1:
        ap.error("--reps must be >= 1")
    cfg = workloads.CONFIGS[a.workload]
    dev = torch.device("cuda", torch.cuda.current_device())
    rigaqep.load()
    sig = torch.from_numpy(workloads.sigma_e(cfg)).to(dev)
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(a.reps)]
    make = lambda: rigaqep.Problem(cfg["ne"], cfg["p"], cfg["block"], sig)  # noqa: E731
    prec = getattr(rigaqep, a.precision)
    opts = EIGS_OPTS.get(a.workload, {})
    extra = {}
    pr = None
    if a.stage in ("assemble", "analyze"):
        for r in range(a.reps):
            if a.stage == "analyze":
                pr = make()
            ev[r][0].record(stream)
            if a.stage == "assemble":
                pr = make()
            else:
                pr.analyze()
            ev[r][1].record(stream)
            torch.cuda.synchronize()
            pr.close()
    else:
        pr = make().analyze()
        if a.stage == "factor":
            for r in range(a.reps):
                ev[r][0].record(stream)
                pr.factor(a.factor_shift, prec)
                ev[r][1].record(stream)
        elif a.stage == "solve":
            pr.factor(a.factor_shift, prec)
            g = torch.Generator(device="cpu").manual_seed(1)
            b = torch.rand(pr.N, dtype=torch.float64, generator=g).to(dev) - 0.5
            x = torch.empty_like(b)
            for r in range(a.reps):
                ev[r][0].record(stream)
                pr.solve(b, out=x)
                ev[r][1].record(stream)
        else:
            for r in range(a.reps):
                ev[r][0].record(stream)
                pr.eigs(cfg["neig"], cfg["shift"], raise_on_noconv=False, precision=prec, **opts)
                ev[r][1].record(stream)
            inf = pr.info()
            extra = {k: inf[k] for k in ("n_apply", "n_restarts", "certified", "fb_ms",
                                         "ritz_ms", "eigs_ms", "factor_ms")}
        torch.cuda.synchronize()
        inf = pr.info()
        extra.update(nnz_L=inf["nnz_L"], nlevels=inf["nlevels"], factor_flops=inf["factor_flops"],
                     precision=a.precision, n_ir=inf["n_ir"], ir_residual=inf["ir_residual"],
                     last_factor_ms=inf["factor_ms"])
        pr.close()
    torch.cuda.synchronize()
    ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    print(json.dumps({"workload": a.workload, "stage": a.stage, "reps": a.reps, "ms": ms,
                      "when": time.strftime("%Y-%m-%dT%H:%M:%S"), **extra}), flush=True)


if __name__ == "__main__":
    main()
