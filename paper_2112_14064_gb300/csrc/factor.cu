// Multifrontal LDL^T of Q(s) = s^2 M + s C + K and supernodal FB solves (FP64).
//
// The paper factorises the shifted quadratic pencil once per shift
// (Algorithm 2, "Factorize Q(s)") with a multifrontal solver and reuses the
// factors in every forward/backward elimination (Section 4.2.2).  For a real
// shift s > 0, Q(s) is SPD, so LDL^T needs no pivoting.
//
// Storage per supernode s with k pivots and u update rows (front order k+u):
//   L panel  (k+u) x k column-major: unit lower pivot block over L21;
//   U block  u x u column-major: the Schur complement handed to the parent.
// The front is the L panel plus the U block (the upper-right part is the
// symmetric counterpart and is never stored).
//
// Factorisation, one launch pair per tree level (all fronts of a level in
// parallel, one CTA per front): (1) zero the front, place the original entries
// of the pivot columns and extend-add the children's U blocks; (2) right-
// looking LDL^T of the k pivot columns with the rank-1 updates applied to the
// pivot block, to L21 and to the U block.
//
// The 32 x 32 diagonal blocks of each unit-lower pivot block are replaced by
// their inverses at the end of the factorisation, so the FB solves apply them
// as small matrix-vector products instead of 32-step substitutions.
//
// FB, two launches per level and sweep.  Forward (leaves first): one CTA per
// front gathers the right-hand side of its pivots and its children's update
// vectors and solves the pivot block (z = L11^{-1} x_s, x_s <- D^{-1} z);
// then the update vectors y_s -= L21 z are formed by CTAs that each own 64
// rows of L21, so large fronts spread over many SMs.  Backward (root first):
// CTAs that each own 32 pivot columns form w = L21^T x_struct (warps split
// the rows, a butterfly reduction gives one column per lane), then one CTA
// per front solves x_s <- L11^{-T} (x_s - w).
#include "internal.h"

namespace rq {
namespace {

struct FrontArgs {
  const int32_t* sptr;
  const int32_t* upd_ptr;
  const int32_t* upd_idx;
  const int32_t* relmap;
  const int32_t* child_ptr;
  const int32_t* child_idx;
  const int32_t* lvl_nodes;
  const int64_t* loff;
  const int64_t* uoff;
  double* Lval;
  double* Uval;
  double* Dinv;
  DevStatus* status;
};

FrontArgs front_args(Problem& P) {
  return FrontArgs{P.sptr.p, P.upd_ptr.p, P.upd_idx.p, P.relmap.p, P.child_ptr.p, P.child_idx.p,
                   P.lvl_nodes.p, P.loff.p, P.uoff.p, P.Lval.p, P.Uval.p, P.Dinv.p, P.status.p};
}

__global__ void k_front_assemble(FrontArgs A, int lvl_begin, const int32_t* rowptr_n,
                                 const int32_t* fpos, const double* Kn, const double* Mn,
                                 const double* Cn, double s2, double s1) {
  int s = A.lvl_nodes[lvl_begin + blockIdx.x];
  int a = A.sptr[s], k = A.sptr[s + 1] - a;
  int u = A.upd_ptr[s + 1] - A.upd_ptr[s];
  int64_t F = k + u;
  double* L = A.Lval + A.loff[s];
  double* U = A.Uval + A.uoff[s];
  for (int64_t i = threadIdx.x; i < F * k; i += blockDim.x) L[i] = 0.0;
  for (int64_t i = threadIdx.x; i < (int64_t)u * u; i += blockDim.x) U[i] = 0.0;
  __syncthreads();
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int t = warp; t < k; t += nw) {
    int j = a + t;
    for (int32_t q = rowptr_n[j] + lane; q < rowptr_n[j + 1]; q += 32) {
      int pos = fpos[q];
      if (pos >= 0) L[pos + F * t] = s2 * Mn[q] + s1 * Cn[q] + Kn[q];
    }
  }
  __syncthreads();
  for (int ci = A.child_ptr[s]; ci < A.child_ptr[s + 1]; ++ci) {
    int c = A.child_idx[ci];
    int uc = A.upd_ptr[c + 1] - A.upd_ptr[c];
    const int32_t* rm = A.relmap + A.upd_ptr[c];
    const double* Uc = A.Uval + A.uoff[c];
    for (int q = warp; q < uc; q += nw) {
      int pc = rm[q];
      for (int r = q + lane; r < uc; r += 32) {
        int pr = rm[r];
        double v = Uc[r + (int64_t)uc * q];
        if (pc < k) L[pr + F * pc] += v;
        else U[(pr - k) + (int64_t)u * (pc - k)] += v;
      }
    }
    __syncthreads();
  }
}

__global__ void k_front_factor(FrontArgs A, int lvl_begin) {
  extern __shared__ double lb[];  // scaled column l (front order)
  __shared__ double dsh;
  int s = A.lvl_nodes[lvl_begin + blockIdx.x];
  int a = A.sptr[s], k = A.sptr[s + 1] - a;
  int u = A.upd_ptr[s + 1] - A.upd_ptr[s];
  int64_t F = k + u;
  double* L = A.Lval + A.loff[s];
  double* U = A.Uval + A.uoff[s];
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int t = 0; t < k; ++t) {
    if (threadIdx.x == 0) {
      double d = L[t + F * t];
      if (!(d > 0.0)) {
        atomicCAS(&A.status->pivot_fail, 0, s + 1);
        d = 1.0;  // keep going with a harmless value; the host reports the failure
      }
      dsh = d;
      L[t + F * t] = 1.0;
      A.Dinv[a + t] = 1.0 / d;
    }
    __syncthreads();
    double d = dsh;
    double rd = 1.0 / d;
    for (int64_t i = t + 1 + threadIdx.x; i < F; i += blockDim.x) {
      double l = L[i + F * t] * rd;
      lb[i] = l;
      L[i + F * t] = l;
    }
    __syncthreads();
    // pivot-block columns c in (t, k): rows i >= c of the L panel
    for (int c = t + 1 + warp; c < k; c += nw) {
      double lc = d * lb[c];
      for (int64_t i = c + lane; i < F; i += 32) L[i + F * c] -= lb[i] * lc;
    }
    // U block columns c' in [0, u): rows i' >= c'
    for (int c = warp; c < u; c += nw) {
      double lc = d * lb[k + c];
      for (int i = c + lane; i < u; i += 32) U[i + (int64_t)u * c] -= lb[k + i] * lc;
    }
    __syncthreads();
  }
  // Replace each 32 x 32 unit-lower diagonal block of L11 by its inverse
  // (lane j: column j by forward substitution), used by the FB solves.
  for (int b0 = warp * 32; b0 < k; b0 += nw * 32) {
    int nb = min(32, k - b0);
    double col[32];
    if (lane < nb) {
      for (int i = 0; i < 32; ++i) col[i] = 0.0;
      col[lane] = 1.0;
      for (int i = lane + 1; i < nb; ++i) {
        double acc = 0.0;
        for (int l = lane; l < i; ++l) acc += L[(b0 + i) + F * (b0 + l)] * col[l];
        col[i] = -acc;
      }
    }
    __syncwarp();
    if (lane < nb)
      for (int i = lane + 1; i < nb; ++i) L[(b0 + i) + F * (b0 + lane)] = col[i];
    __syncwarp();
  }
}

struct FBArgs {
  const int32_t* sptr;
  const int32_t* upd_ptr;
  const int32_t* upd_idx;
  const int32_t* relmap;
  const int32_t* child_ptr;
  const int32_t* child_idx;
  const int32_t* lvl_nodes;
  const int64_t* loff;
  const double* Lval;
  const double* Dinv;
  double* yvec;
  double* zbuf;    // unscaled forward solution of the pivot rows
  double* wbuf;    // L21^T x_struct of the pivot rows (backward)
  const int4* fwd_items;  // (front, first row of L21, rows)
  const int4* bwd_items;  // (front, first pivot column, columns)
};

FBArgs fb_args(Problem& P) {
  return FBArgs{P.sptr.p,  P.upd_ptr.p, P.upd_idx.p, P.relmap.p, P.child_ptr.p,
                P.child_idx.p, P.lvl_nodes.p, P.loff.p, P.Lval.p, P.Dinv.p,
                P.yvec.p, P.zbuf.p, P.wbuf.p, (const int4*)P.fwd_items.p,
                (const int4*)P.bwd_items.p};
}

// Butterfly transpose-reduction of 32 per-lane accumulators: afterwards lane
// l holds the warp-wide sum of acc[l] in acc[0] (31 additions per lane).
__device__ __forceinline__ double warp_transpose_reduce(double (&acc)[32], int lane) {
#pragma unroll
  for (int o = 16, len = 32; o > 0; o >>= 1, len >>= 1) {
    bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < len / 2; ++i) {
      double send = up ? acc[i] : acc[i + len / 2];
      double keep = up ? acc[i + len / 2] : acc[i];
      acc[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return acc[0];
}

// Forward, pivot rows of one front per CTA: gather the right-hand side and the
// children's update vectors, then z = L11^{-1} x_s in 32-row blocks (the
// diagonal blocks hold their inverses), x_s <- D^{-1} z.
__global__ void k_fb_fwd_tri(FBArgs A, int lvl_begin, double* x) {
  extern __shared__ double xs[];
  int s = A.lvl_nodes[lvl_begin + blockIdx.x];
  int a = A.sptr[s], k = A.sptr[s + 1] - a;
  int u = A.upd_ptr[s + 1] - A.upd_ptr[s];
  int64_t F = k + u;
  const double* L = A.Lval + A.loff[s];
  double* ys = A.yvec + A.upd_ptr[s];
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int t = threadIdx.x; t < k; t += blockDim.x) xs[t] = x[a + t];
  for (int i = threadIdx.x; i < u; i += blockDim.x) ys[i] = 0.0;
  __syncthreads();
  for (int ci = A.child_ptr[s]; ci < A.child_ptr[s + 1]; ++ci) {
    int c = A.child_idx[ci];
    int uc = A.upd_ptr[c + 1] - A.upd_ptr[c];
    const int32_t* rm = A.relmap + A.upd_ptr[c];
    const double* yc = A.yvec + A.upd_ptr[c];
    for (int r = threadIdx.x; r < uc; r += blockDim.x) {
      int pos = rm[r];
      double v = yc[r];
      if (pos < k) xs[pos] += v;
      else ys[pos - k] += v;
    }
    __syncthreads();
  }
  for (int b0 = 0; b0 < k; b0 += 32) {
    int nb = min(32, k - b0);
    if (warp == 0) {
      // z_b = inv(L_bb) x_b, lane = row.  Loads are unconditional (clamped
      // to the block) so they issue together; out-of-range terms are zeroed.
      int rr = min(lane, nb - 1);
      const double* row = L + (b0 + rr) + F * b0;
      double v[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) v[c] = row[F * min(c, nb - 1)];
      double a0 = 0.0, a1 = 0.0;
#pragma unroll
      for (int c = 0; c < 32; c += 2) {
        a0 += (c <= lane ? v[c] : 0.0) * xs[b0 + min(c, nb - 1)];
        a1 += (c + 1 <= lane ? v[c + 1] : 0.0) * xs[b0 + min(c + 1, nb - 1)];
      }
      __syncwarp();
      if (lane < nb) xs[b0 + lane] = a0 + a1;
    }
    __syncthreads();
    for (int i = b0 + nb + threadIdx.x; i < k; i += blockDim.x) {
      const double* row = L + i + F * b0;
      double acc = 0.0;
      if (nb == 32) {
        double v[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) v[c] = row[F * c];
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
#pragma unroll
        for (int c = 0; c < 32; c += 4) {
          a0 += v[c] * xs[b0 + c];
          a1 += v[c + 1] * xs[b0 + c + 1];
          a2 += v[c + 2] * xs[b0 + c + 2];
          a3 += v[c + 3] * xs[b0 + c + 3];
        }
        acc = (a0 + a1) + (a2 + a3);
      } else {
        for (int c = 0; c < nb; ++c) acc += row[F * c] * xs[b0 + c];
      }
      xs[i] -= acc;
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < k; t += blockDim.x) {
    A.zbuf[a + t] = xs[t];
    x[a + t] = xs[t] * A.Dinv[a + t];
  }
}

// Forward, update rows: y_s[r] -= L21[r, :] z_s for one block of rows.
__global__ void k_fb_fwd_gemv(FBArgs A, int item_begin) {
  int4 it = A.fwd_items[item_begin + blockIdx.x];
  int s = it.x;
  int a = A.sptr[s], k = A.sptr[s + 1] - a;
  int u = A.upd_ptr[s + 1] - A.upd_ptr[s];
  int64_t F = k + u;
  const double* L = A.Lval + A.loff[s];
  double* ys = A.yvec + A.upd_ptr[s];
  extern __shared__ double zs[];
  for (int t = threadIdx.x; t < k; t += blockDim.x) zs[t] = A.zbuf[a + t];
  __syncthreads();
  int r = it.y + threadIdx.x;
  if (threadIdx.x >= it.z) return;
  const double* row = L + k + r;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  int t = 0;
  for (; t + 8 <= k; t += 8) {
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q & 3] += row[F * (t + q)] * zs[t + q];
  }
  for (; t < k; ++t) acc[0] += row[F * t] * zs[t];
  ys[r] -= (acc[0] + acc[1]) + (acc[2] + acc[3]);
}

// Backward, w = L21^T x_struct for a block of <= 32 pivot columns: warps split
// the update rows, lanes run along a column, butterfly to one column per lane.
__global__ void k_fb_bwd_gemv(FBArgs A, int item_begin, const double* x) {
  int4 it = A.bwd_items[item_begin + blockIdx.x];
  int s = it.x, c0 = it.y, nc = it.z;
  int a = A.sptr[s], k = A.sptr[s + 1] - a;
  int u = A.upd_ptr[s + 1] - A.upd_ptr[s];
  int64_t F = k + u;
  const double* L = A.Lval + A.loff[s];
  const int32_t* st = A.upd_idx + A.upd_ptr[s];
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double acc[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) acc[c] = 0.0;
  for (int i = warp * 32 + lane; i < u; i += nw * 32) {
    double xv = x[st[i]];
    const double* row = L + k + i + F * c0;
    double v[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) v[c] = row[F * min(c, nc - 1)];
#pragma unroll
    for (int c = 0; c < 32; ++c) acc[c] += v[c] * xv;
  }
  double v = warp_transpose_reduce(acc, lane);
  __shared__ double red[8][32];
  red[warp][lane] = v;
  __syncthreads();
  if (threadIdx.x < nc) {
    double sum = 0.0;
    for (int w = 0; w < nw; ++w) sum += red[w][threadIdx.x];
    A.wbuf[a + c0 + threadIdx.x] = sum;
  }
}

// Backward, pivot rows of one front per CTA: x_s <- L11^{-T} (x_s - w), last
// 32-block first; each block subtracts the already solved rows below it
// (butterfly column dots) and applies the transposed inverse diagonal block.
__global__ void k_fb_bwd_tri(FBArgs A, int lvl_begin, double* x, double sigma, const double* vu,
                             double* ru, double* rl) {
  extern __shared__ double xs[];
  __shared__ double red[8][32];
  int s = A.lvl_nodes[lvl_begin + blockIdx.x];
  int a = A.sptr[s], k = A.sptr[s + 1] - a;
  int u = A.upd_ptr[s + 1] - A.upd_ptr[s];
  int64_t F = k + u;
  const double* L = A.Lval + A.loff[s];
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int t = threadIdx.x; t < k; t += blockDim.x)
    xs[t] = x[a + t] - (u > 0 ? A.wbuf[a + t] : 0.0);
  __syncthreads();
  int nblk = (k + 31) / 32;
  for (int bi = nblk - 1; bi >= 0; --bi) {
    int b0 = bi * 32;
    int nb = min(32, k - b0);
    int r0 = b0 + nb;
    if (r0 < k) {
      double acc[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) acc[c] = 0.0;
      for (int i = r0 + warp * 32 + lane; i < k; i += nw * 32) {
        double xv = xs[i];
        const double* row = L + i + F * b0;
        double v[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) v[c] = row[F * min(c, nb - 1)];
#pragma unroll
        for (int c = 0; c < 32; ++c) acc[c] += v[c] * xv;
      }
      double v = warp_transpose_reduce(acc, lane);
      red[warp][lane] = v;
      __syncthreads();
      if (threadIdx.x < nb) {
        double sum = 0.0;
        for (int w = 0; w < nw; ++w) sum += red[w][threadIdx.x];
        xs[b0 + threadIdx.x] -= sum;
      }
      __syncthreads();
    }
    if (warp == 0) {
      // x_b = inv(L_bb)^T x_b, lane = column (clamped unconditional loads)
      const double* colp = L + b0 + F * (b0 + min(lane, nb - 1));
      double v[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) v[i] = colp[min(i, nb - 1)];
      double a0 = 0.0, a1 = 0.0;
#pragma unroll
      for (int i = 0; i < 32; i += 2) {
        a0 += (i >= lane && i < nb ? v[i] : 0.0) * xs[b0 + min(i, nb - 1)];
        a1 += (i + 1 >= lane && i + 1 < nb ? v[i + 1] : 0.0) * xs[b0 + min(i + 1, nb - 1)];
      }
      __syncwarp();
      if (lane < nb) xs[b0 + lane] = a0 + a1;
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < k; t += blockDim.x) {
    double v = xs[t];
    x[a + t] = v;
    if (ru) {
      ru[a + t] = -v;
      rl[a + t] = sigma * (-v) + vu[a + t];
    }
  }
}

__global__ void k_gather(const int32_t* idx, const double* src, double* dst, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[idx[i]];
}

__global__ void k_scatter(const int32_t* idx, const double* src, double* dst, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) dst[idx[i]] = src[i];
}

}  // namespace

void factor_configure(size_t smem_max) {
  int v = (int)smem_max;
  if (smem_max <= 48 * 1024) return;
  RQ_CUDA(cudaFuncSetAttribute(k_front_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, v));
  RQ_CUDA(cudaFuncSetAttribute(k_fb_fwd_tri, cudaFuncAttributeMaxDynamicSharedMemorySize, v));
  RQ_CUDA(cudaFuncSetAttribute(k_fb_fwd_gemv, cudaFuncAttributeMaxDynamicSharedMemorySize, v));
  RQ_CUDA(cudaFuncSetAttribute(k_fb_bwd_tri, cudaFuncAttributeMaxDynamicSharedMemorySize, v));
}

void launch_factor(Problem& P, double sigma) {
  Plan& L = P.plan;
  cudaStream_t s = P.stream;
  FrontArgs A = front_args(P);
  for (int l = 0; l < L.nlevels; ++l) {
    int b = L.lvl_ptr[l], cnt = L.lvl_ptr[l + 1] - b;
    k_front_assemble<<<cnt, 256, 0, s>>>(A, b, P.rowptr_n.p, P.fpos.p, P.Kn.p, P.Mn.p, P.Cn.p,
                                         sigma * sigma, sigma);
    RQ_CUDA(cudaGetLastError());
    size_t smem = sizeof(double) * (size_t)P.lvl_maxF[l];
    k_front_factor<<<cnt, 256, smem, s>>>(A, b);
    RQ_CUDA(cudaGetLastError());
    P.launches += 2;
  }
}

void fb_plan(Problem& P) {
  Plan& L = P.plan;
  std::vector<int32_t> fwd, bwd;
  P.fwd_lvl.assign(L.nlevels + 1, 0);
  P.bwd_lvl.assign(L.nlevels + 1, 0);
  for (int l = 0; l < L.nlevels; ++l) {
    for (int q = L.lvl_ptr[l]; q < L.lvl_ptr[l + 1]; ++q) {
      int s = L.lvl_nodes[q];
      int k = L.sptr[s + 1] - L.sptr[s], u = L.upd_ptr[s + 1] - L.upd_ptr[s];
      for (int r = 0; r < u; r += 64) fwd.insert(fwd.end(), {s, r, std::min(64, u - r), 0});
      if (u > 0)
        for (int c = 0; c < k; c += 32) bwd.insert(bwd.end(), {s, c, std::min(32, k - c), 0});
    }
    P.fwd_lvl[l + 1] = (int32_t)(fwd.size() / 4);
    P.bwd_lvl[l + 1] = (int32_t)(bwd.size() / 4);
  }
  P.fwd_items.upload(fwd, P.stream);
  P.bwd_items.upload(bwd, P.stream);
  P.zbuf.alloc(L.N);
  P.wbuf.alloc(L.N);
}

void launch_fb(Problem& P, double* xn, double sigma, const double* vu, double* ru, double* rl) {
  Plan& L = P.plan;
  cudaStream_t s = P.stream;
  FBArgs A = fb_args(P);
  for (int l = 0; l < L.nlevels; ++l) {
    int b = L.lvl_ptr[l], cnt = L.lvl_ptr[l + 1] - b;
    k_fb_fwd_tri<<<cnt, 256, sizeof(double) * (size_t)P.lvl_maxK[l], s>>>(A, b, xn);
    RQ_CUDA(cudaGetLastError());
    ++P.launches;
    int ib = P.fwd_lvl[l], ic = P.fwd_lvl[l + 1] - ib;
    if (ic > 0) {
      k_fb_fwd_gemv<<<ic, 64, sizeof(double) * (size_t)P.lvl_maxK[l], s>>>(A, ib);
      RQ_CUDA(cudaGetLastError());
      ++P.launches;
    }
  }
  for (int l = L.nlevels - 1; l >= 0; --l) {
    int b = L.lvl_ptr[l], cnt = L.lvl_ptr[l + 1] - b;
    int ib = P.bwd_lvl[l], ic = P.bwd_lvl[l + 1] - ib;
    if (ic > 0) {
      k_fb_bwd_gemv<<<ic, 256, 0, s>>>(A, ib, xn);
      RQ_CUDA(cudaGetLastError());
      ++P.launches;
    }
    k_fb_bwd_tri<<<cnt, 256, sizeof(double) * (size_t)P.lvl_maxK[l], s>>>(A, b, xn, sigma, vu, ru, rl);
    RQ_CUDA(cudaGetLastError());
    ++P.launches;
  }
}

void launch_gather(const int32_t* idx, const double* src, double* dst, int64_t n, int32_t ld_in,
                   int32_t ncol, cudaStream_t s) {
  for (int c = 0; c < ncol; ++c) {
    k_gather<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(idx, src + (int64_t)c * ld_in,
                                                          dst + (int64_t)c * n, n);
    RQ_CUDA(cudaGetLastError());
  }
}

void launch_scatter(const int32_t* idx, const double* src, double* dst, int64_t n, cudaStream_t s) {
  k_scatter<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(idx, src, dst, n);
  RQ_CUDA(cudaGetLastError());
}

}  // namespace rq
