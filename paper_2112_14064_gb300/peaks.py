"""Measured arithmetic peaks of the GPU for the roofline denominators.

The front factorisation runs in FP64 (FP64 pipe), FP32 (SIMT) or on the
tensor cores in TF32 / BF16; the bench quotes each kernel against the rate
measured here rather than a nominal figure.  Each rate is the best of
`reps` timed dense products C = A B of n x n matrices through torch.matmul
(cuBLAS), 2 n^3 flops each, timed with CUDA events on the current stream
after two warm-up products.

    python -m paper_2112_14064_gb300.peaks [--n 8192] [--reps 5]

Prints one JSON object: {"fp64_tflops", "fp32_tflops", "tf32_tflops",
"bf16_tflops", "n", "reps", "device", "sm_count"}.
"""
import argparse
import json

import torch


def _rate(dtype, n, reps, tf32=False):
    torch.backends.cuda.matmul.allow_tf32 = tf32
    g = torch.Generator(device="cuda").manual_seed(1)
    a = torch.rand((n, n), device="cuda", dtype=dtype, generator=g)
    b = torch.rand((n, n), device="cuda", dtype=dtype, generator=g)
    for _ in range(2):
        c = a @ b
    torch.cuda.synchronize()
    best = float("inf")
    s = torch.cuda.current_stream()
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        c = a @ b
        e1.record(s)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) * 1e-3)
    del c
    torch.backends.cuda.matmul.allow_tf32 = False
    return 2.0 * n ** 3 / best / 1e12


def measure(n=8192, reps=5):
    props = torch.cuda.get_device_properties(0)
    return {
        "fp64_tflops": _rate(torch.float64, n, reps),
        "fp32_tflops": _rate(torch.float32, n, reps, tf32=False),
        "tf32_tflops": _rate(torch.float32, n, reps, tf32=True),
        "bf16_tflops": _rate(torch.bfloat16, n, reps),
        "n": n, "reps": reps, "device": props.name, "sm_count": props.multi_processor_count,
    }


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--reps", type=int, default=5)
    a = ap.parse_args()
    print(json.dumps(measure(a.n, a.reps)), flush=True)
