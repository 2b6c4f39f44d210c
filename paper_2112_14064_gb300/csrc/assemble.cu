// Element-batched Gauss-quadrature assembly of K, M and C (FP64).
//
// Space: tensor-product B-splines on the unit square (paper Section 3.1),
// identity geometric map, rIGA or IGA knots (Sections 3.2-3.3).  For a
// tensor-product function pair on an axis-aligned element the 2-D Gauss sum
// factorises exactly into 1-D sums:
//   int_e B_a B_b      = mx_e(ax,bx) * my_e(ay,by)
//   int_e grad.grad    = kx_e * my_e + mx_e * ky_e
// with mx_e(a,b) = sum_q w_q N_a(x_q) N_b(x_q), kx_e with derivatives.
// Step 1 computes those 1-D element integrals for every element and local
// pair (one thread each, Cox-de Boor evaluated at the Gauss points); step 2
// forms each CSR entry by summing over the elements shared by its two
// functions (one thread per row, no atomics, deterministic):
//   M_ij = sum_e mx my,  K_ij = sum_e (kx my + mx ky),  C_ij = sum_e sigma_e mx my.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

namespace rq {
namespace {

struct Tables {
  const int* knots;      // numerators over ne
  const int* first_fn;   // first full function of element ex
  const int* elo;        // element range of DOF d
  const int* ehi;
  const double* gx;      // Gauss points on [-1, 1]
  const double* gw;      // Gauss weights
  int ne, p, nq, n1;
};

// Values and first derivatives of the p+1 B-splines that do not vanish on
// knot span s (full functions s-p .. s) at x.  Cox-de Boor (paper Eqs.
// BasisFunBi0/BasisFunBip) on the triangular table of non-zero functions:
// degree q keeps functions s-q..s; every denominator t_{i+q}-t_i or
// t_{i+q+1}-t_{i+1} that is used spans the non-empty span s, so none is zero.
__device__ void basis_on_span(const int* knots, double inv_ne, int s, int p, double x,
                              double* N, double* dN) {
  double prev[kMaxP + 1], cur[kMaxP + 1];
  prev[0] = 1.0;
  auto t = [&](int i) { return (double)knots[i] * inv_ne; };
  for (int q = 1; q <= p; ++q) {
    for (int r = 0; r <= q; ++r) {
      int i = s - q + r;
      double v = 0.0;
      if (r >= 1) v += (x - t(i)) / (t(i + q) - t(i)) * prev[r - 1];
      if (r <= q - 1) v += (t(i + q + 1) - x) / (t(i + q + 1) - t(i + 1)) * prev[r];
      cur[r] = v;
    }
    if (q == p) {
      for (int r = 0; r <= p; ++r) {
        int i = s - p + r;
        double d = 0.0;
        if (r >= 1) d += p / (t(i + p) - t(i)) * prev[r - 1];
        if (r <= p - 1) d -= p / (t(i + p + 1) - t(i + 1)) * prev[r];
        N[r] = cur[r];
        dN[r] = d;
      }
      return;
    }
    for (int r = 0; r <= q; ++r) prev[r] = cur[r];
  }
}

// m1[ex][a][b], k1[ex][a][b]: 1-D element mass/stiffness integrals.
__global__ void k_element_1d(Tables T, double* m1, double* k1) {
  int np1 = T.p + 1;
  int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t total = (int64_t)T.ne * np1 * np1;
  if (tid >= total) return;
  int b = tid % np1;
  int a = (tid / np1) % np1;
  int ex = tid / (np1 * np1);
  double inv_ne = 1.0 / T.ne;
  int s = T.first_fn[ex] + T.p;
  double N[kMaxP + 1], dN[kMaxP + 1];
  double mm = 0.0, kk = 0.0;
  for (int q = 0; q < T.nq; ++q) {
    double x = (ex + 0.5 * (T.gx[q] + 1.0)) * inv_ne;
    double w = T.gw[q] * 0.5 * inv_ne;
    basis_on_span(T.knots, inv_ne, s, T.p, x, N, dN);
    mm += w * N[a] * N[b];
    kk += w * dN[a] * dN[b];
  }
  m1[tid] = mm;
  k1[tid] = kk;
}

__global__ void k_assemble_rows(Tables T, const int32_t* rowptr, const int32_t* col,
                                const double* m1, const double* k1, const double* sig,
                                double* K, double* M, double* C) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t Nn = (int64_t)T.n1 * T.n1;
  if (r >= Nn) return;
  int n1 = T.n1, np1 = T.p + 1;
  int ix = r % n1, iy = r / n1;
  for (int32_t q = rowptr[r]; q < rowptr[r + 1]; ++q) {
    int c = col[q];
    int jx = c % n1, jy = c / n1;
    int ex0 = max(T.elo[ix], T.elo[jx]), ex1 = min(T.ehi[ix], T.ehi[jx]);
    int ey0 = max(T.elo[iy], T.elo[jy]), ey1 = min(T.ehi[iy], T.ehi[jy]);
    // The shared elements are the product [ex0, ex1) x [ey0, ey1), so the
    // element sums of M and K factor into 1-D sums:
    //   M = (sum_x m_x)(sum_y m_y),  K = (sum_x k_x)(sum_y m_y) + (sum_x m_x)(sum_y k_y);
    // C = sum_y m_y sum_x sigma(x, y) m_x keeps its double sum.
    double mxs[kMaxP + 1];
    double Mx = 0.0, Kx = 0.0;
    for (int ex = ex0; ex < ex1; ++ex) {
      int g0 = T.first_fn[ex];
      int ax = ix + 1 - g0, bx = jx + 1 - g0;
      double mx = m1[((int64_t)ex * np1 + ax) * np1 + bx];
      mxs[ex - ex0] = mx;
      Mx += mx;
      Kx += k1[((int64_t)ex * np1 + ax) * np1 + bx];
    }
    double My = 0.0, Ky = 0.0, sc = 0.0;
    for (int ey = ey0; ey < ey1; ++ey) {
      int f0 = T.first_fn[ey];
      int ay = iy + 1 - f0, by = jy + 1 - f0;
      double my = m1[((int64_t)ey * np1 + ay) * np1 + by];
      My += my;
      Ky += k1[((int64_t)ey * np1 + ay) * np1 + by];
      const double* sg = sig + ex0 + (int64_t)T.ne * ey;
      double in = 0.0;
      for (int ex = ex0; ex < ex1; ++ex) in += sg[ex - ex0] * mxs[ex - ex0];
      sc += my * in;
    }
    K[q] = Kx * My + Mx * Ky;
    M[q] = Mx * My;
    C[q] = sc;
  }
}

__global__ void k_permute(const int32_t* map, const double* a, const double* b, const double* c,
                          double* an, double* bn, double* cn, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t o = map[i];
  an[i] = a[o];
  bn[i] = b[o];
  cn[i] = c[o];
}

// max-row-sum norms; non-negative doubles order like their bit patterns
// max-row-sum norms of K, M, C (out[0..2]) and the largest entries of K and
// M (out[3..4]); non-negative doubles compare like their bit patterns
__global__ void k_row_norms(const int32_t* rowptr, const double* K, const double* M,
                            const double* C, int64_t N, unsigned long long* out) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (r < N) {
    for (int32_t q = rowptr[r]; q < rowptr[r + 1]; ++q) {
      s[0] += fabs(K[q]);
      s[1] += fabs(M[q]);
      s[2] += fabs(C[q]);
      s[3] = fmax(s[3], fabs(K[q]));
      s[4] = fmax(s[4], fabs(M[q]));
    }
  }
  for (int t = 0; t < 5; ++t) {
    double v = s[t];
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out + t, (unsigned long long)__double_as_longlong(v));
  }
}

// Gauss-Legendre nodes and weights by Newton's method on P_n (host).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = pk;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = pk;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

}  // namespace

void launch_assemble(Problem& P) {
  Plan& L = P.plan;
  cudaStream_t s = P.stream;
  std::vector<double> gx, gw;
  gauss_legendre(L.nq, gx, gw);
  DBuf<int> knots, elo, ehi;
  DBuf<double> dgx, dgw;
  DBuf<int>& first_fn = P.first_fn;
  DBuf<double>& m1 = P.m1;
  DBuf<double>& k1 = P.k1;
  knots.upload(L.sp.knots, s);
  first_fn.upload(L.sp.first_fn, s);
  elo.upload(L.sp.elo, s);
  ehi.upload(L.sp.ehi, s);
  dgx.upload(gx, s);
  dgw.upload(gw, s);
  int np1 = L.p + 1;
  int64_t ntab = (int64_t)L.ne * np1 * np1;
  m1.alloc(ntab);
  k1.alloc(ntab);
  Tables T{knots.p, first_fn.p, elo.p, ehi.p, dgx.p, dgw.p, L.ne, L.p, L.nq, L.n1};
  k_element_1d<<<(unsigned)((ntab + 255) / 256), 256, 0, s>>>(T, m1.p, k1.p);
  RQ_CUDA(cudaGetLastError());
  P.K.alloc(L.nnz);
  P.M.alloc(L.nnz);
  P.C.alloc(L.nnz);
  k_assemble_rows<<<(unsigned)((L.N + 127) / 128), 128, 0, s>>>(T, P.rowptr.p, P.col.p, m1.p, k1.p,
                                                                 P.sigma_e.p, P.K.p, P.M.p, P.C.p);
  RQ_CUDA(cudaGetLastError());
  RQ_CUDA(cudaStreamSynchronize(s));  // temporaries are freed on return
}

void launch_norms(Problem& P) {
  DBuf<unsigned long long> out;
  out.alloc(5);
  RQ_CUDA(cudaMemsetAsync(out.p, 0, 5 * sizeof(unsigned long long), P.stream));
  int64_t N = P.plan.N;
  k_row_norms<<<(unsigned)((N + 255) / 256), 256, 0, P.stream>>>(P.rowptr.p, P.K.p, P.M.p, P.C.p, N,
                                                                  out.p);
  RQ_CUDA(cudaGetLastError());
  unsigned long long h[5];
  RQ_CUDA(cudaMemcpyAsync(h, out.p, sizeof(h), cudaMemcpyDeviceToHost, P.stream));
  RQ_CUDA(cudaStreamSynchronize(P.stream));
  double d[5];
  for (int t = 0; t < 5; ++t) std::memcpy(&d[t], &h[t], sizeof(double));
  P.info.norm_K = d[0];
  P.info.norm_M = d[1];
  P.info.norm_C = d[2];
  P.maxabs_K = d[3];
  P.maxabs_M = d[4];
}

// ND-ordered CSR of the pattern, one warp per ND row j (the original row
// perm[j]): its columns renumbered by iperm and sorted (each entry's rank
// among the row's distinct keys gives its slot), the original slot of each
// entry, and the row of each lower-triangle entry (column i >= j) in the
// front of j's supernode: i - a for the supernode's own pivots, k + (place of
// i in its structure) otherwise, -1 above the diagonal.  err: 1 a row longer
// than kNdMaxRow, 2 an entry outside the front (a broken symbolic phase).
constexpr int kNdMaxRow = 256;
constexpr int kNdWarps = 8;

__global__ void __launch_bounds__(32 * kNdWarps) k_nd_csr(
    const int32_t* perm, const int32_t* iperm, const int32_t* rowptr, const int32_t* col,
    const int32_t* rowptr_n, const int32_t* sptr, int nsuper, const int32_t* upd_ptr,
    const int32_t* upd_idx, int64_t N, int32_t* col_n, int32_t* slot_map, int32_t* fpos,
    int32_t* err) {
  __shared__ int32_t keys[kNdWarps][kNdMaxRow];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t j = (int64_t)blockIdx.x * kNdWarps + warp;
  if (j >= N) return;   // whole warps
  const int32_t o = perm[j], q0 = rowptr[o], n = rowptr[o + 1] - q0;
  if (n > kNdMaxRow) {
    if (lane == 0) atomicExch(err, 1);
    return;
  }
  for (int e = lane; e < n; e += 32) keys[warp][e] = iperm[col[q0 + e]];
  __syncwarp();
  // supernode of row j: the last s with sptr[s] <= j
  int lo = 0, hi = nsuper - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (sptr[mid] <= j) lo = mid;
    else hi = mid - 1;
  }
  const int a = sptr[lo], e1 = sptr[lo + 1], k = e1 - a;
  const int32_t* ps = upd_idx + upd_ptr[lo];
  const int u = upd_ptr[lo + 1] - upd_ptr[lo];
  const int32_t base = rowptr_n[j];
  for (int e = lane; e < n; e += 32) {
    const int32_t key = keys[warp][e];
    int rank = 0;
    for (int f = 0; f < n; ++f) rank += keys[warp][f] < key ? 1 : 0;
    const int32_t t = base + rank;
    col_n[t] = key;
    slot_map[t] = q0 + e;
    int32_t fp = -1;
    if (key >= j) {
      if (key < e1) {
        fp = key - a;
      } else {
        int l2 = 0, h2 = u;   // first structure entry >= key
        while (l2 < h2) {
          const int mid = (l2 + h2) >> 1;
          if (ps[mid] < key) l2 = mid + 1;
          else h2 = mid;
        }
        if (l2 < u && ps[l2] == key) fp = k + l2;
        else atomicExch(err, 2);
      }
    }
    fpos[t] = fp;
  }
}

void launch_nd_csr(Problem& P, int32_t* err) {
  const Plan& L = P.plan;
  P.col_n.alloc(L.nnz);
  P.slot_map.alloc(L.nnz);
  P.fpos.alloc(L.nnz);
  k_nd_csr<<<(unsigned)((L.N + kNdWarps - 1) / kNdWarps), 32 * kNdWarps, 0, P.stream>>>(
      P.perm.p, P.iperm.p, P.rowptr.p, P.col.p, P.rowptr_n.p, P.sptr.p, L.nsuper, P.upd_ptr.p,
      P.upd_idx.p, L.N, P.col_n.p, P.slot_map.p, P.fpos.p, err);
  RQ_CUDA(cudaGetLastError());
}

void launch_permute_values(Problem& P) {
  int64_t n = P.plan.nnz;
  P.Kn.alloc(n);
  P.Mn.alloc(n);
  P.Cn.alloc(n);
  k_permute<<<(unsigned)((n + 255) / 256), 256, 0, P.stream>>>(P.slot_map.p, P.K.p, P.M.p, P.C.p,
                                                               P.Kn.p, P.Mn.p, P.Cn.p, n);
  RQ_CUDA(cudaGetLastError());
}

// SELL-32: thread (slice s, lane l) writes row 32 s + l's entries at
// off + 32 k + l; slots past the row's end (and rows past N) get column 0 and
// zero values.
__global__ void k_sell_fill(const int32_t* rowptr, const int32_t* col, const double* Mn,
                            const double* Cn, const int32_t* off, int64_t ns, int64_t N,
                            int32_t* scol, double* sM, double* sC) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t sl = r >> 5;
  if (sl >= ns) return;
  const int l = (int)(r & 31);
  const int32_t o0 = off[sl], w = (off[sl + 1] - o0) >> 5;
  const int32_t q0 = r < N ? rowptr[r] : 0, n = r < N ? rowptr[r + 1] - q0 : 0;
  for (int k = 0; k < w; ++k) {
    const int64_t e = o0 + 32 * (int64_t)k + l;
    scol[e] = k < n ? col[q0 + k] : 0;
    sM[e] = k < n ? Mn[q0 + k] : 0.0;
    sC[e] = k < n ? Cn[q0 + k] : 0.0;
  }
}

void launch_sell(Problem& P) {
  const Plan& L = P.plan;
  const int64_t N = L.N, ns = (N + 31) / 32;
  std::vector<int32_t>& off = P.sell_off_h;
  off.assign(ns + 1, 0);
  for (int64_t sl = 0; sl < ns; ++sl) {
    int32_t w = 0;
    for (int64_t r = 32 * sl; r < std::min(N, 32 * sl + 32); ++r)
      w = std::max(w, L.rowptr_n[r + 1] - L.rowptr_n[r]);
    off[sl + 1] = off[sl] + 32 * w;
  }
  P.sell_off.upload(off, P.stream);
  P.sell_col.alloc(off[ns]);
  P.sell_M.alloc(off[ns]);
  P.sell_C.alloc(off[ns]);
  k_sell_fill<<<(unsigned)((32 * ns + 255) / 256), 256, 0, P.stream>>>(
      P.rowptr_n.p, P.col_n.p, P.Mn.p, P.Cn.p, P.sell_off.p, ns, N, P.sell_col.p, P.sell_M.p,
      P.sell_C.p);
  RQ_CUDA(cudaGetLastError());
}

}  // namespace rq
