"""Throughput of the rIGA shift-and-invert QEP solve on GB300.

One step = the whole path on the 256 x 256-element, p = 3 rIGA mesh with
C^0 lines every 16 elements (82,369 DOFs): Gauss-quadrature assembly of
K, M, C, the symbolic phase, the multifrontal factorisation and the
Krylov-Schur eigensolve of the 20 eigenpairs nearest the target 500
(FP64).  The spectral shift is placed inside the spectrum region (shift 0,
56 candidates, Krylov dimension 96) and the selection nearest the target is
certified; a pair counts only when its backward error is <= 1e-10 and the
selection is certified.

Further legs of the same JSON line (each its own workload, timed the same
way): the same step with FP32, split-TF32 and split-BF16 fronts and FP64
refinement (`mixed`); the p = 4, 512 x 512 lognormal-damping workload in
FP64 and with tensor-core fronts (`workload_mixed`); the p = 3, 512 x 512
differentiation workload with all 262,144 damping gradients (`workload_grad`);
the same 256 x 256 mesh with maximum-continuity IGA against rIGA (`iga`);
the complex shift i sqrt(500) and the undamped slice [500, 1000) of the
headline mesh (`variants`); and the 64-problem batch (`batch`).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun every rank solves its own copy
(the single-QEP path does not shard: replicas), value = all pairs / max time.
"""
import os

os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")   # the CPU oracle runs single-threaded
os.environ.setdefault("OMP_NUM_THREADS", "1")

import argparse
import hashlib
import json
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "p3_256_b16"
TARGET_KW = dict(m=96, shift=0.0, ncand=56)
ETA_MAX = 1e-10
METRIC = "eigenpairs/s at rel. residual <= 1e-10 (FP64)"
UNIT = "eigenpairs/s"
BATCH_KW = dict(shift=0.0, ncand=24, m=48, seed=1)   # in-region solve shared by a problem's 4 targets
BATCH_TIMED = 2   # timed steps of the batch leg
FP64_NOMINAL_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12   # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-workload leg")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision leg")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the 512^2 workload legs and the IGA comparison")
    return ap.parse_args()


class Clocks(threading.Thread):
    """nvidia-smi samples (SM clock, max clock, throttle reasons) while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        super().__init__(daemon=True)
        self.index = str(index)
        self.rows = []
        self.proc = None

    def run(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            for line in self.proc.stdout:
                parts = [p.strip() for p in line.split(",")]
                if parts and parts[0] == self.index:
                    self.rows.append(parts)
        except Exception:
            pass

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if len(r) > 5 + i and r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(self.rows)}


def fb_source_hash():
    """sha256 of the FB kernels' source text (the sweep kernels and their
    launchers in factor.cu): the committed DRAM counters stay valid while it
    is unchanged."""
    src = open(os.path.join(ROOT, "paper_2112_14064_gb300", "csrc", "factor.cu")).read()
    a = src.index("// Forward sweep, one work item")
    b = src.index("__global__ void k_gather")
    c = src.index("void launch_fb_t(")
    d = src.index("\n}\n", src.index("void launch_fb(")) + 3
    return hashlib.sha256((src[a:b] + src[c:d]).encode()).hexdigest()


def fb_traffic(nnz_L):
    """DRAM bytes per FB solve from the committed ncu summary, if the FB
    kernels are unchanged since it was taken (source hash); else None."""
    path = os.path.join(ROOT, "profiles", "fb_solve_traffic.json")
    try:
        rec = json.load(open(path))
        if rec.get("fb_kernels_sha256") != fb_source_hash() or rec.get("nnz_L") != nnz_L:
            return None
        return rec["dram_bytes_per_solve"]
    except Exception:
        return None


def oracle_sample(cfg, sig, v1):
    """Time the FP64 CPU oracle as it stands on one full solve of the
    workload: its own assembly, symbolic phase, factorisation at the shift
    and the whole Krylov-Schur eigensolve (same target, shift, candidates and
    Krylov dimension as the GPU step).  Returns (pairs/s, seconds,
    description)."""
    from oracle.assemble import assemble
    from oracle.nd import symbolic
    from oracle.multifrontal import factorize
    from oracle import qep
    t0 = time.perf_counter()
    A = assemble(cfg["ne"], cfg["p"], cfg["block"], sig)
    sym = symbolic(A.n1, A.space.c0_dofs, cfg["p"], A.indptr, A.indices)
    F = factorize(sym, A.Q(TARGET_KW["shift"]))
    t1 = time.perf_counter()
    r = qep.eigs(A.K, A.C, A.M, TARGET_KW["shift"], cfg["neig"], TARGET_KW["m"], F.solve, v1,
                 target=cfg["shift"], ncand=TARGET_KW["ncand"], sigma_min=sig.min())
    t2 = time.perf_counter()
    pairs = int((r.eta <= ETA_MAX).sum()) if r.certified else 0
    desc = (f"one full oracle solve of the workload: assemble+symbolic+factor {t1 - t0:.1f} s, "
            f"Krylov-Schur {t2 - t1:.1f} s ({r.n_apply} applies, {r.n_restarts} restarts), "
            f"{pairs} certified pairs; single thread (host has {os.cpu_count()} cores)")
    return pairs / (t2 - t0), t2 - t0, desc


def run_reference(args):
    import torch  # noqa: F401  (torch is imported by the GPU arm too; keeps timings comparable)
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2112_14064_gb300 import workloads
    cfg = workloads.CONFIGS[WORKLOAD]
    sig = workloads.sigma_e(cfg)
    N = (cfg["ne"] + cfg["p"] - 2 + (cfg["ne"] // cfg["block"] - 1) * (cfg["p"] - 1)) ** 2
    v1 = workloads.start_vector(1, 2 * N)
    # warm-up: the checker on its tiny configuration (imports, allocator)
    tiny = workloads.CONFIGS["tiny"]
    from oracle.assemble import assemble
    for _ in range(args.warmup):
        assemble(tiny["ne"], tiny["p"], tiny["block"], workloads.sigma_e(tiny))
    vals, secs, desc = [], [], ""
    for _ in range(args.steps):
        v, t, desc = oracle_sample(cfg, sig, v1)
        vals.append(v)
        secs.append(t)
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean(secs)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "ne": cfg["ne"], "p": cfg["p"],
                       "block": cfg["block"], "target": cfg["shift"], "neig": cfg["neig"],
                       **TARGET_KW},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": desc, "host_cores": os.cpu_count()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batch_leg(rank, world, barrier):
    """The batched workload: 64 independent problems (ne 32..256, p 2..5,
    blocks of 8 or 16, sigma_e ~ U[0.05, 2]) with 4 targets each, 8 pairs
    per target; problems are dealt to ranks round-robin (no exchange).  One
    step = assemble every problem on its own stream + rigaqep_batch_eigs
    (analyze, factor, in-region eigensolve shared by the 4 targets,
    selection and extraction per target) + release; host-timed around a
    device synchronisation (the work spans many streams and the call returns
    its results to the host).  One warm-up step and BATCH_TIMED timed steps;
    `seconds` is their mean."""
    import torch
    from paper_2112_14064_gb300 import rigaqep, workloads
    cfgs = workloads.batch_problems()
    mine = [i for i in range(len(cfgs)) if i % world == rank]
    sig = {i: torch.from_numpy(workloads.sigma_e(cfgs[i])).cuda() for i in mine}
    streams = [torch.cuda.Stream() for _ in mine]

    def step():
        probs = [rigaqep.Problem(cfgs[i]["ne"], cfgs[i]["p"], cfgs[i]["block"], sig[i],
                                 stream=streams[q]) for q, i in enumerate(mine)]
        jobs = [dict(problem=q, neig=cfgs[i]["neig"], target=t, **BATCH_KW)
                for q, i in enumerate(mine) for t in cfgs[i]["shifts"]]
        res = rigaqep.batch_eigs(probs, jobs, raise_on_error=False)
        torch.cuda.synchronize()
        conv = sum(int((r["eta"] <= ETA_MAX).sum()) for r in res if r["status"] in (0, 7))
        cert = sum(int((r["eta"] <= ETA_MAX).sum()) for r in res
                   if r["status"] in (0, 7) and r["certified"])
        for pr in probs:
            pr.close()
        return len(jobs), conv, cert

    step()
    barrier()
    per = []
    for _ in range(BATCH_TIMED):
        t0 = time.perf_counter()
        njobs, conv, cert = step()
        torch.cuda.synchronize()
        per.append(time.perf_counter() - t0)
    return dict(problems=len(mine), jobs=njobs, pairs_converged=conv, pairs_certified=cert,
                seconds=sum(per) / len(per), seconds_each=per)


def measured_fp64_peak(dev, n=4096, reps=3):
    """FP64 dense-product rate of this GPU (TFLOP/s): best of `reps`
    torch.matmul (cuBLAS DGEMM) of n x n matrices, CUDA events."""
    import torch
    a = torch.rand((n, n), dtype=torch.float64, device=dev)
    b = torch.rand((n, n), dtype=torch.float64, device=dev)
    c = a @ b
    torch.cuda.synchronize()
    best = float("inf")
    st = torch.cuda.current_stream()
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        c = a @ b
        e1.record(st)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) * 1e-3)
    del a, b, c
    return 2.0 * n ** 3 / best / 1e12


def _timed(step, n, flush, stream):
    """n steps, each after an L2 flush, CUDA events on the stream around each."""
    import torch
    times, outs = [], []
    for i in range(n):
        flush.fill_(float(i))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        outs.append(step())
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return times, outs


def _rel_diffs(ref, got):
    """Per computed eigenvalue: relative distance to the nearest reference value."""
    return [float(np.min(np.abs(ref - v)) / abs(v)) for v in got]


def _solve_step(cfg, sig_d, kw, prec, v1_d=None):
    """One assemble + analyze + factor + eigs step; returns (lam, eta, info)."""
    from paper_2112_14064_gb300 import rigaqep
    pr = rigaqep.Problem(cfg["ne"], cfg["p"], cfg["block"], sig_d).analyze()
    lam, X, eta, nconv, st = pr.eigs(cfg["neig"], cfg["shift"], v1=v1_d, raise_on_noconv=False,
                                     precision=getattr(rigaqep, prec), **kw)
    inf = pr.info()
    pr.close()
    return lam, eta, inf


def _leg_entry(times, outs, lam64, certified_only=True):
    lam, eta, inf = outs[-1]
    good = 0
    for l_, e_, i_ in outs:
        ok = int((e_ <= ETA_MAX).sum().item())
        good += ok if (i_["certified"] == 1 or not certified_only) else 0
    ent = {"value": 1e3 * good / sum(times), "unit": UNIT,
           "ms_per_step": sum(times) / len(times), "steps": len(times),
           "certified": int(inf["certified"]), "cert_margin": inf["cert_margin"],
           "factor_ms": inf["factor_ms"],
           "factor_tflops": inf["factor_flops_exact"] / (inf["factor_ms"] * 1e-3) / 1e12,
           "factor_tflops_executed": inf["factor_flops"] / (inf["factor_ms"] * 1e-3) / 1e12,
           "refinement_steps": inf["n_ir"], "probe_residual": inf["ir_residual"],
           "n_apply": inf["n_apply"], "fb_ms": inf["fb_ms"], "eigs_ms": inf["eigs_ms"],
           "max_eta": float(eta.max().item())}
    if lam64 is not None:
        d = _rel_diffs(lam64, lam.cpu().numpy())
        ent["rel_eigenvalue_diff_vs_fp64"] = d
        ent["max_rel_eigenvalue_diff_vs_fp64"] = max(d)
    return ent


def precision_leg(cfg, kw, sig_d, v1_d, lam64, flush, stream, barrier, steps=2):
    """The bench step with FP32 (SIMT), split-TF32 and split-BF16 (tcgen05)
    fronts, every solve refined in FP64; eigenvalues against the FP64 step's
    result by result."""
    out = {"workload": WORKLOAD, "note": "same step as the headline with low-precision fronts "
           "and FP64-refined solves; value counts certified pairs with eta <= 1e-10"}
    for prec in ("FP32_IR", "TF32_IR", "BF16_IR"):
        _solve_step(cfg, sig_d, kw, prec, v1_d)
        barrier()
        times, outs = _timed(lambda: _solve_step(cfg, sig_d, kw, prec, v1_d), steps, flush, stream)
        out[prec] = _leg_entry(times, outs, lam64)
    return out


WORKLOAD_MIXED_KW = dict(m=96, shift=0.0, ncand=88, seed=1)
WORKLOAD_GRAD_KW = dict(m=96, shift=0.0, ncand=80, seed=1)


def workload_mixed_leg(flush, stream, barrier):
    """p = 4, 512 x 512, blocks of 32, lognormal damping (median 0.5,
    log-std 1), 20 pairs nearest the target 2000: FP64 fronts and split
    TF32 / BF16 tensor-core fronts with FP64 refinement, eigenvalues against
    the FP64 result.  With 88 candidates (m = 96) the selection at this
    target is not certified (the damping spread needs ~400 candidates), so
    the value counts converged pairs with eta <= 1e-10 and `certified` is
    reported."""
    import torch
    from paper_2112_14064_gb300 import workloads
    cfg = workloads.CONFIGS["p4_512_b32"]
    sig_d = torch.from_numpy(workloads.sigma_e(cfg)).cuda()
    out = {"workload": "p4_512_b32", "N": None, "solve": WORKLOAD_MIXED_KW,
           "target": cfg["shift"], "neig": cfg["neig"],
           "value_counts": "converged pairs with eta <= 1e-10 (selection not certified)"}
    lam64 = None
    for prec in ("FP64", "TF32_IR", "BF16_IR"):
        _solve_step(cfg, sig_d, WORKLOAD_MIXED_KW, prec)
        barrier()
        times, outs = _timed(lambda: _solve_step(cfg, sig_d, WORKLOAD_MIXED_KW, prec), 1, flush,
                             stream)
        out[prec] = _leg_entry(times, outs, lam64, certified_only=False)
        out["N"] = outs[-1][2]["N"]
        if prec == "FP64":
            lam64 = outs[-1][0].cpu().numpy()
    return out


def workload_grad_leg(flush, stream, barrier):
    """p = 3, 512 x 512, blocks of 16, sigma_e ~ U[0.1, 1], 20 pairs nearest
    800 (certified): one step = assemble + analyze + factor + eigs + the
    gradients of the 20 eigenvalues with respect to all 262,144 sigma_e, in
    FP64 and with the split-TF32 forward pass."""
    import torch
    from paper_2112_14064_gb300 import rigaqep, workloads
    cfg = workloads.CONFIGS["p3_512_b16"]
    sig_d = torch.from_numpy(workloads.sigma_e(cfg)).cuda()
    ne2 = cfg["ne"] ** 2
    out = {"workload": "p3_512_b16", "solve": WORKLOAD_GRAD_KW, "target": cfg["shift"],
           "neig": cfg["neig"], "gradients_per_step": cfg["neig"] * ne2}

    def step(prec):
        pr = rigaqep.Problem(cfg["ne"], cfg["p"], cfg["block"], sig_d).analyze()
        lam, X, eta, nconv, st = pr.eigs(cfg["neig"], cfg["shift"], raise_on_noconv=False,
                                         precision=getattr(rigaqep, prec), **WORKLOAD_GRAD_KW)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        G = pr.grad_damping(lam, X)
        e1.record(stream)
        inf = pr.info()
        pr.close()
        return lam, eta, inf, (e0, e1), G

    lam64 = None
    for prec in ("FP64", "TF32_IR"):
        step(prec)
        barrier()
        times, outs = _timed(lambda: step(prec), 2, flush, stream)
        lam, eta, inf, (e0, e1), G = outs[-1]
        ent = _leg_entry(times, [(o[0], o[1], o[2]) for o in outs], lam64)
        ent["adjoint_ms"] = e0.elapsed_time(e1)
        ent["gradients_per_s"] = 1e3 * cfg["neig"] * ne2 / (sum(times) / len(times))
        ent["adjoint_gradients_per_s"] = 1e3 * cfg["neig"] * ne2 / ent["adjoint_ms"]
        ent["adjoint_gb_per_s"] = (16.0 * cfg["neig"] * (outs[-1][2]["N"] + 2 * ne2)
                                   / (ent["adjoint_ms"] * 1e-3) / 1e9)
        out[prec] = ent
        if prec == "FP64":
            lam64 = lam.cpu().numpy()
    return out


def iga_leg(inf_riga, riga_ms, flush, stream, barrier):
    """The headline step on the same mesh with maximum-continuity IGA (C^2,
    no C^0 separators) against rIGA (blocks of 16): factor flops (exact),
    factor time, factor entries (the FB bytes), eigensolve time and
    eigenpairs/s; the analogue of the paper's rIGA-vs-IGA comparison
    (Table 2) for this scalar problem."""
    import torch
    from paper_2112_14064_gb300 import workloads
    cfg = workloads.CONFIGS["p3_256_iga"]
    sig_d = torch.from_numpy(workloads.sigma_e(cfg)).cuda()
    _solve_step(cfg, sig_d, TARGET_KW, "FP64")
    barrier()
    times, outs = _timed(lambda: _solve_step(cfg, sig_d, TARGET_KW, "FP64"), 2, flush, stream)
    ent = _leg_entry(times, outs, None)
    inf = outs[-1][2]
    ent.update(N=inf["N"], nnz_L_exact=inf["nnz_L_exact"], factor_flops_exact=inf["factor_flops_exact"],
               fb_ms_per_solve=inf["fb_ms"] / max(1, inf["n_apply"]))
    r = {"N": inf_riga["N"], "nnz_L_exact": inf_riga["nnz_L_exact"],
         "factor_flops_exact": inf_riga["factor_flops_exact"], "factor_ms": inf_riga["factor_ms"],
         "fb_ms_per_solve": inf_riga["fb_ms"] / max(1, inf_riga["n_apply"]),
         "eigs_ms": inf_riga["eigs_ms"], "ms_per_step": riga_ms}
    return {"workload": "p3_256_iga (C^2) against p3_256_b16 (rIGA, blocks of 16)",
            "iga": ent, "riga": r,
            "improvement_riga_over_iga": {
                "factor_flops": inf["factor_flops_exact"] / r["factor_flops_exact"],
                "factor_time": ent["factor_ms"] / r["factor_ms"],
                "factor_entries": inf["nnz_L_exact"] / r["nnz_L_exact"],
                "fb_time": ent["fb_ms_per_solve"] / r["fb_ms_per_solve"],
                "eigs_time": ent["eigs_ms"] / r["eigs_ms"],
                "step_time": ent["ms_per_step"] / r["ms_per_step"]}}


def variants_leg(flush, stream, barrier):
    """The headline mesh (p = 3, 256 x 256, blocks of 16) solved two other
    ways: the 20 pairs nearest the complex shift i sqrt(500) through the
    complex symmetric factor of Q(s) and the real operator Re((A - sB)^-1 B)
    (one step = analyze + complex factor + eigs), and every undamped
    eigenvalue mu = omega^2 of K x = mu M x in [500, 1000) with its count
    certified by two inertias (one step = analyze + two indefinite factors +
    shift-invert Lanczos)."""
    import torch
    from paper_2112_14064_gb300 import rigaqep, workloads
    cfg = workloads.CONFIGS[WORKLOAD]
    sig_d = torch.from_numpy(workloads.sigma_e(cfg)).cuda()
    shift = 1j * np.sqrt(500.0)

    def cstep():
        pr = rigaqep.Problem(cfg["ne"], cfg["p"], cfg["block"], sig_d).analyze()
        lam, X, eta, nconv, st = pr.eigs(cfg["neig"], 1.0, m=96, shift=shift, seed=1,
                                         raise_on_noconv=False)
        inf = pr.info()
        pr.close()
        return lam, eta, inf

    def ustep():
        pr = rigaqep.Problem(cfg["ne"], cfg["p"], cfg["block"], sig_d).analyze()
        out = pr.eigs_undamped(500.0, 1000.0, seed=1)
        pr.close()
        return out

    cstep()
    barrier()
    times, outs = _timed(cstep, 2, flush, stream)
    lam, eta, inf = outs[-1]
    good = sum(int((e <= ETA_MAX).sum().item()) for _, e, _ in outs)
    cx = {"shift": "i*sqrt(500)", "neig": cfg["neig"], "value": 1e3 * good / sum(times),
          "unit": UNIT, "ms_per_step": sum(times) / len(times), "steps": len(times),
          "factor_ms": inf["factor_ms"], "fb_ms": inf["fb_ms"], "n_apply": inf["n_apply"],
          "eigs_ms": inf["eigs_ms"], "max_eta": float(eta.max().item()),
          "max_rel_imag_offset": float(np.max(np.abs(lam.cpu().numpy().imag - np.sqrt(500.0)))
                                       / np.sqrt(500.0))}
    ustep()
    barrier()
    times, outs = _timed(ustep, 2, flush, stream)
    mu, X, res, count, cert = outs[-1]
    good = sum(int((r <= ETA_MAX).sum().item()) if c == 1 else 0 for _, _, r, _, c in outs)
    ud = {"interval": [500.0, 1000.0], "count": int(count), "certified": int(cert),
          "value": 1e3 * good / sum(times), "unit": "undamped eigenpairs/s",
          "ms_per_step": sum(times) / len(times), "steps": len(times),
          "max_residual": float(res.max().item()) if len(mu) else 0.0}
    return {"workload": WORKLOAD, "complex_shift": cx, "undamped_slice": ud}


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2112_14064_gb300 import rigaqep, workloads

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    rigaqep.load()

    cfg = workloads.CONFIGS[WORKLOAD]
    sig_h = workloads.sigma_e(cfg)
    sig_d = torch.from_numpy(sig_h).to(dev)
    probe = rigaqep.symbolic_host(cfg["ne"], cfg["p"], cfg["block"])
    N = len(probe["perm"])
    v1_h = workloads.start_vector(1, 2 * N)
    v1_d = torch.from_numpy(v1_h).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    neig, target = cfg["neig"], cfg["shift"]

    def step(sig, v1):
        pr = rigaqep.Problem(cfg["ne"], cfg["p"], cfg["block"], sig).analyze()
        lam, X, eta, nconv, st = pr.eigs(neig, target, v1=v1, raise_on_noconv=False, **TARGET_KW)
        inf = pr.info()
        good = (eta <= ETA_MAX).sum() if inf["certified"] == 1 else torch.zeros((), device=dev)
        pr.close()
        return lam, X, eta, good, inf

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for i in range(args.warmup):
        step(sig_d, v1_d)
    barrier()

    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.5)
    stream = torch.cuda.current_stream()
    times, pairs, infos = [], 0, []
    barrier()
    for i in range(args.steps):
        flush.fill_(float(i))                     # L2 flush between timed steps
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lam, X, eta, good, inf = step(sig_d, v1_d)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        pairs += int(good.item())
        infos.append(inf)
    barrier()
    clocks.stop()
    total_ms = float(sum(times))

    # end to end through host buffers: pinned inputs in, results out, every step
    sig_pin = torch.from_numpy(sig_h).pin_memory()
    v1_pin = torch.from_numpy(v1_h).pin_memory()
    lam_pin = torch.empty((neig, 2), dtype=torch.float64).pin_memory()
    X_pin = torch.empty((neig, N, 2), dtype=torch.float64).pin_memory()
    eta_pin = torch.empty(neig, dtype=torch.float64).pin_memory()
    e2e_ms, e2e_pairs = [], 0
    barrier()
    for i in range(args.steps):
        flush.fill_(float(i))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sig_dev = sig_pin.to(dev, non_blocking=True)
        v1_dev = v1_pin.to(dev, non_blocking=True)
        lam, X, eta, good, inf = step(sig_dev, v1_dev)
        lam_pin.copy_(torch.view_as_real(lam), non_blocking=True)
        X_pin.copy_(torch.view_as_real(X), non_blocking=True)
        eta_pin.copy_(eta, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
        e2e_pairs += int(good.item())
    barrier()

    # one more (untimed) step, synchronised after every stage, for the breakdown
    stages = {}
    barrier()
    t0 = time.perf_counter()
    pr = rigaqep.Problem(cfg["ne"], cfg["p"], cfg["block"], sig_d)
    torch.cuda.synchronize()
    stages["assemble_ms"] = 1e3 * (time.perf_counter() - t0)
    t0 = time.perf_counter()
    pr.analyze()
    torch.cuda.synchronize()
    stages["analyze_ms"] = 1e3 * (time.perf_counter() - t0)
    t0 = time.perf_counter()
    pr.eigs(neig, target, v1=v1_d, raise_on_noconv=False, **TARGET_KW)
    torch.cuda.synchronize()
    stages["factor_and_eigs_ms"] = 1e3 * (time.perf_counter() - t0)
    t0 = time.perf_counter()
    pr.close()
    torch.cuda.synchronize()
    stages["release_ms"] = 1e3 * (time.perf_counter() - t0)

    batch = None if args.no_batch else batch_leg(rank, world, barrier)

    # precision, workload and discretisation legs (each its own workload)
    legs = {}
    if not args.no_mixed:
        legs["mixed"] = precision_leg(cfg, TARGET_KW, sig_d, v1_d, lam.cpu().numpy(), flush,
                                      stream, barrier, steps=2)
    if not args.no_workloads:
        legs["workload_mixed"] = workload_mixed_leg(flush, stream, barrier)
        legs["workload_grad"] = workload_grad_leg(flush, stream, barrier)
        legs["iga"] = iga_leg(infos[-1], total_ms / args.steps, flush, stream, barrier)
        legs["variants"] = variants_leg(flush, stream, barrier)

    # max over ranks
    t = torch.tensor([total_ms, float(sum(e2e_ms))], dtype=torch.float64, device=dev)
    pr_t = torch.tensor([float(pairs), float(e2e_pairs)], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(pr_t, op=dist.ReduceOp.SUM)
    total_ms, e2e_total = float(t[0]), float(t[1])
    all_pairs, all_e2e_pairs = float(pr_t[0]), float(pr_t[1])

    inf = infos[-1]
    fb_avg_s = inf["fb_ms"] / max(1, inf["n_apply"]) / 1e3
    nnz_L = inf["nnz_L"]
    nnz_exact = inf["nnz_L_exact"]
    # algorithmic work of one solve: every structurally non-zero entry of L
    # once forward and once backward (one FMA and 8 bytes each), plus the
    # right-hand side and solution vectors
    fb_flops = 4.0 * nnz_exact
    fb_bytes = 16.0 * nnz_exact + 32.0 * inf["N"]
    achieved_tf = fb_flops / fb_avg_s / 1e12
    fp64_peak = measured_fp64_peak(dev)
    traffic = fb_traffic(nnz_L)
    line = {
        "metric": METRIC, "value": 1e3 * all_pairs / total_ms, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded sigma_e ~ U[0.1, 1] per element, splitmix64 start vector)",
        "config": {"workload": WORKLOAD, "ne": cfg["ne"], "p": cfg["p"], "block": cfg["block"],
                   "N": N, "target": target, "neig": neig, **TARGET_KW,
                   "parallelism": f"replicas x{world}",
                   "l2": "256 MB buffer written between timed steps"},
        "roofline": {"kernel": "FB solve (forward + backward substitution kernels)",
                     "bound": "alu", "achieved": achieved_tf, "peak": fp64_peak,
                     "unit": "TFLOP/s", "frac": achieved_tf / fp64_peak,
                     "peak_source": "FP64 DGEMM (torch.matmul, 4096^3) measured in this run",
                     "peak_nominal": FP64_NOMINAL_TFLOPS,
                     "traffic": traffic, "algorithmic_bytes": fb_bytes,
                     "algorithmic_flops": fb_flops, "nnz_L_exact": nnz_exact,
                     "nnz_L_stored": nnz_L, "avg_launch_us": fb_avg_s * 1e6,
                     "hbm_frac": fb_bytes / fb_avg_s / 1e9 / _hbm_peak()},
        "factor": {"tflops": inf["factor_flops_exact"] / (inf["factor_ms"] * 1e-3) / 1e12,
                   "tflops_executed": inf["factor_flops"] / (inf["factor_ms"] * 1e-3) / 1e12,
                   "ms": inf["factor_ms"], "flops_exact": inf["factor_flops_exact"],
                   "flops_executed": inf["factor_flops"],
                   "frac_of_fp64_peak": inf["factor_flops_exact"] / (inf["factor_ms"] * 1e-3)
                   / 1e12 / fp64_peak},
        "solve": {"n_apply": inf["n_apply"], "n_restarts": inf["n_restarts"],
                  "certified": inf["certified"], "eigs_ms": inf["eigs_ms"],
                  "fb_ms": inf["fb_ms"], "ritz_ms": inf["ritz_ms"]},
        "stages_host_ms": stages,
        "clocks": clocks.summary(),
        "e2e": {"value": 1e3 * all_e2e_pairs / e2e_total, "unit": UNIT,
                "h2d_bytes_per_step": 8 * (cfg["ne"] ** 2) + 16 * N,
                "d2h_bytes_per_step": 16 * neig + 16 * N * neig + 8 * neig},
        "gpu_launches": int(sum(i["n_launches"] + 4 for i in infos)),
    }
    line.update(legs)
    if batch is not None:
        bt = torch.tensor([batch["seconds"], batch["jobs"], batch["pairs_converged"],
                           batch["pairs_certified"], batch["problems"]], dtype=torch.float64,
                          device=dev)
        if world > 1:
            mx = bt[:1].clone()
            dist.all_reduce(mx, op=dist.ReduceOp.MAX)
            dist.all_reduce(bt, op=dist.ReduceOp.SUM)
            bt[0] = mx[0]
        secs = float(bt[0])
        line["batch"] = {
            "workload": "64 problems (ne 32-256, p 2-5, blocks 8/16, sigma_e ~ U[0.05, 2]), "
                        "4 targets in [10, 5000] each, 8 pairs per target",
            "solve": BATCH_KW, "problems": int(bt[4]), "jobs": int(bt[1]),
            "pairs_converged": int(bt[2]), "pairs_certified": int(bt[3]), "seconds": secs,
            "converged_pairs_per_s": float(bt[2]) / secs,
            "certified_pairs_per_s": float(bt[3]) / secs,
            "timing": "host clock around a device synchronisation, 1 warm-up + %d timed steps "
                      "(mean)" % BATCH_TIMED, "seconds_each_rank0": batch["seconds_each"]}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, secs, desc = oracle_sample(cfg, sig_h, v1_h)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": desc, "host_cores": os.cpu_count()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _hbm_peak():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except Exception:
        return 6800.0


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
