"""Throughput of the rIGA shift-and-invert QEP solve on GB300.

One step = the whole path on the 256 x 256-element, p = 3 rIGA mesh with
C^0 lines every 16 elements (82,369 DOFs): Gauss-quadrature assembly of
K, M, C, the symbolic phase, the multifrontal factorisation and the
Krylov-Schur eigensolve of the 20 eigenpairs nearest the target 500
(FP64).  The spectral shift is placed inside the spectrum region (shift 0,
56 candidates, Krylov dimension 96) and the selection nearest the target is
certified; a pair counts only when its backward error is <= 1e-10 and the
selection is certified.

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
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12   # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-workload leg")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision leg")
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
    """sha256 of the FB kernels' source text (the two sweep kernels and their
    launcher in factor.cu): the committed DRAM counters stay valid while it
    is unchanged."""
    src = open(os.path.join(ROOT, "paper_2112_14064_gb300", "csrc", "factor.cu")).read()
    a = src.index("// Forward sweep, one work item")
    b = src.index("__global__ void k_gather")
    c = src.index("void launch_fb(")
    d = src.index("\n}\n", c) + 3
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


def oracle_sample(cfg, sig, v1, n_apply_full):
    """Time the FP64 CPU oracle on a bounded sample of the workload: its own
    assembly, symbolic phase, factorisation at the shift and one Krylov-Schur
    cycle (m operator applications with CGS2); extrapolate one full solve as
    setup + n_apply_full / m cycles.  Returns (pairs/s, seconds, description)."""
    from oracle.assemble import assemble
    from oracle.nd import symbolic
    from oracle.multifrontal import factorize
    from oracle import qep
    t0 = time.perf_counter()
    A = assemble(cfg["ne"], cfg["p"], cfg["block"], sig)
    sym = symbolic(A.n1, A.space.c0_dofs, cfg["p"], A.indptr, A.indices)
    F = factorize(sym, A.Q(TARGET_KW["shift"]))
    t1 = time.perf_counter()
    qep.eigs(A.K, A.C, A.M, TARGET_KW["shift"], cfg["neig"], TARGET_KW["m"], F.solve, v1,
             max_restarts=0, target=cfg["shift"], ncand=TARGET_KW["ncand"], sigma_min=sig.min())
    t2 = time.perf_counter()
    cycle = (t2 - t1) / TARGET_KW["m"]
    full = (t1 - t0) + n_apply_full * cycle
    desc = (f"oracle assemble+symbolic+factor ({t1 - t0:.1f} s) and one Krylov-Schur cycle of "
            f"{TARGET_KW['m']} applies ({t2 - t1:.1f} s) on the full workload; one solve "
            f"extrapolated to the GPU's {n_apply_full} applies = {full:.1f} s")
    return cfg["neig"] / full, t2 - t0, desc


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
    n_apply_full = int(os.environ.get("RIGAQEP_REF_APPLIES", "167"))   # the GPU arm's applies
    vals, secs, desc = [], [], ""
    for _ in range(args.steps):
        v, t, desc = oracle_sample(cfg, sig, v1, n_apply_full)
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
                             "sample": desc},
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
    device synchronisation (the work spans many streams).  One warm-up step
    and one timed step."""
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
    t0 = time.perf_counter()
    njobs, conv, cert = step()
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    return dict(problems=len(mine), jobs=njobs, pairs_converged=conv, pairs_certified=cert,
                seconds=secs)


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

    # mixed precision: the same step with FP32 fronts and FP64-refined solves,
    # its eigenvalues against the FP64 step's
    mixed = None
    if not args.no_mixed:
        lam64 = lam.cpu().numpy()

        def step_mixed():
            pr = rigaqep.Problem(cfg["ne"], cfg["p"], cfg["block"], sig_d).analyze()
            lm, Xm, em, nc, st = pr.eigs(neig, target, v1=v1_d, raise_on_noconv=False,
                                         precision=rigaqep.FP32_IR, **TARGET_KW)
            im = pr.info()
            gm = (em <= ETA_MAX).sum() if im["certified"] == 1 else torch.zeros((), device=dev)
            pr.close()
            return lm, gm, im

        step_mixed()
        barrier()
        mt, mp, minf, lmx = [], 0, None, None
        for i in range(2):
            flush.fill_(float(i))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lmx, gm, minf = step_mixed()
            e1.record(stream)
            torch.cuda.synchronize()
            mt.append(e0.elapsed_time(e1))
            mp += int(gm.item())
        lm_h = lmx.cpu().numpy()
        diff = max(float(np.min(np.abs(lam64 - v)) / abs(v)) for v in lm_h)
        mixed = {"precision": "FP32 fronts and sweeps, FP64-refined solves",
                 "value": 1e3 * mp / sum(mt), "unit": UNIT, "ms_per_step": sum(mt) / len(mt),
                 "factor_ms": minf["factor_ms"],
                 "factor_tflops": minf["factor_flops"] / (minf["factor_ms"] * 1e-3) / 1e12,
                 "refinement_steps": minf["n_ir"], "probe_residual": minf["ir_residual"],
                 "fb_ms": minf["fb_ms"], "n_apply": minf["n_apply"],
                 "max_rel_eigenvalue_diff_vs_fp64": diff, "steps": len(mt)}

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
    fb_flops = 4.0 * nnz_L                       # every factor entry: one FMA forward, one backward
    fb_bytes = 16.0 * nnz_L + 32.0 * inf["N"]    # factor read twice + rhs/solution vectors
    achieved_tf = fb_flops / fb_avg_s / 1e12
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
                     "bound": "alu", "achieved": achieved_tf, "peak": FP64_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved_tf / FP64_PEAK_TFLOPS,
                     "traffic": traffic, "algorithmic_bytes": fb_bytes,
                     "avg_launch_us": fb_avg_s * 1e6,
                     "hbm_frac": fb_bytes / fb_avg_s / 1e9 / _hbm_peak()},
        "factor": {"tflops": inf["factor_flops"] / (inf["factor_ms"] * 1e-3) / 1e12,
                   "ms": inf["factor_ms"], "flops": inf["factor_flops"]},
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
    if mixed is not None:
        line["mixed"] = mixed
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
            "timing": "host clock around a device synchronisation, 1 warm-up + 1 timed step"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, secs, desc = oracle_sample(cfg, sig_h, v1_h, inf["n_apply"])
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": desc}
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
