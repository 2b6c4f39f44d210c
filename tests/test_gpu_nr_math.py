"""The Newton-Raphson FP64 reciprocal, quotient and square root used by the
Ritz step, against CUDA's own FP64 operators (at most 2 ulp apart)."""
import os
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = r'''
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <cmath>
#include "nr_math.cuh"
__global__ void k(const double* a, const double* b, double* out, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[6 * i + 0] = rq::rcp_nr(b[i]);
  out[6 * i + 1] = 1.0 / b[i];
  out[6 * i + 2] = rq::div_nr(a[i], b[i]);
  out[6 * i + 3] = a[i] / b[i];
  double x = fabs(b[i]);
  out[6 * i + 4] = rq::sqrt_nr(x);
  out[6 * i + 5] = sqrt(x);
}
int main() {
  const int n = 1 << 16;
  double *ha = new double[n], *hb = new double[n], *ho = new double[6 * n];
  uint64_t z = 88172645463325252ull;
  for (int i = 0; i < n; ++i) {
    z ^= z << 13; z ^= z >> 7; z ^= z << 17;
    double u = (double)(z >> 11) * 0x1.0p-53;
    z ^= z << 13; z ^= z >> 7; z ^= z << 17;
    double w = (double)(z >> 11) * 0x1.0p-53;
    ha[i] = (u - 0.5) * pow(10.0, 40.0 * w - 20.0);
    hb[i] = (w - 0.5) * pow(10.0, 64.0 * u - 32.0);
    if (hb[i] == 0.0) hb[i] = 1.0;
  }
  double *da, *db, *dout;
  cudaMalloc(&da, n * 8); cudaMalloc(&db, n * 8); cudaMalloc(&dout, 6 * n * 8);
  cudaMemcpy(da, ha, n * 8, cudaMemcpyHostToDevice);
  cudaMemcpy(db, hb, n * 8, cudaMemcpyHostToDevice);
  k<<<(n + 255) / 256, 256>>>(da, db, dout, n);
  if (cudaMemcpy(ho, dout, 6 * n * 8, cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
  long long worst[3] = {0, 0, 0};
  for (int i = 0; i < n; ++i)
    for (int f = 0; f < 3; ++f) {
      int64_t p, q;
      memcpy(&p, &ho[6 * i + 2 * f], 8);
      memcpy(&q, &ho[6 * i + 2 * f + 1], 8);
      long long d = llabs((long long)(p - q));
      if (d > worst[f]) worst[f] = d;
    }
  printf("%lld %lld %lld\n", worst[0], worst[1], worst[2]);
  return 0;
}
'''


def test_newton_raphson_helpers_within_2_ulp(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    src = tmp_path / "nr.cu"
    src.write_text(SRC)
    exe = tmp_path / "nr"
    inc = os.path.join(ROOT, "paper_2112_14064_gb300", "csrc")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-I", inc,
                    str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    rcp, div, sq = (int(v) for v in out)
    assert rcp <= 2 and div <= 2 and sq <= 2, (rcp, div, sq)
