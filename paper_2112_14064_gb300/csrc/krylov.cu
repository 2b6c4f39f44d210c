// Shift-and-invert Krylov-Schur on the linearised QEP (FP64), device side.
//
// Linearisation (paper Eq. Linearization): A = [[0, I], [-K, -C]],
// B = diag(I, M).  Operator (Eq. BlockOperatorVector):
//   r_u = -Q(s)^{-1} (s M v_u + C v_u + M v_l),   r_l = s r_u + v_u.
// B-inner product (Section 4.2.1): <x, y>_B = x_u^T y_u + x_l^T M y_l.
// Arnoldi step j (Algorithms 1 and 2) with classical Gram-Schmidt applied
// twice (CGS2): h = V^T B r, r -= V h (twice), h_{j+1,j} = ||r||_B,
// v_{j+1} = r / h_{j+1,j}.  Ritz step and truncation: ritz.cu.
//
// The Krylov basis lives in the nested-dissection order of the factor, so
// no permutation is needed per step: V is (3 Np) x (m+1), column-major,
// column c = [v_u (Np); v_l (Np); w = M v_l (Np)] with Np = N rounded up to
// a whole TMA tile of rows (zero pad).  Keeping the B-image w of every basis
// vector (formed by the B-norm kernel, which computes M v_l anyway) turns the
// projections into h = V_u^T r_u + W^T r_l (M is symmetric), so that neither
// Gram-Schmidt pass needs a sparse product; the restart rotates W with V.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include <complex>

#include "internal.h"
#include "tma.cuh"

namespace rq {

size_t ritz_smem(int m);
void launch_ritz(const double* H, double* Hnew, double* Q, double* Y, RitzOut* out, int m, int neig,
                 int kwant, int final_pass, int lock, double sigma, double tol, double tscale,
                 cudaStream_t s);

namespace {

// Sparse products over the SELL-32 copy of the pattern (slot k of row
// 32 s + l at off[s] + 32 k + l; padded slots hold column 0 and zero values).
// kSplit warps share a slice: warp t takes slots k = t mod kSplit of all 32
// rows, so that every load of the pattern and the values is coalesced, each
// FP64 instruction does 32 rows' work (on this GPU every FP64 warp
// instruction costs 64 cycles of its sub-partition's pipe whatever its active
// lanes), and there are kSplit threads per row to keep loads in flight.  The
// partial sums meet in shared memory.  A block of 256 threads covers two
// slices.
constexpr int kSplit = 4;
constexpr int kSellBlock = 256;
constexpr int kSlicesPerBlock = kSellBlock / 32 / kSplit;
constexpr int kSellUnroll = 4;   // slots of a thread's row loaded together
static_assert(kSlicesPerBlock >= 1, "a block covers whole slices");
// sum of the kSplit partial sums of row `lane` of the slice whose first warp is w0
__device__ __forceinline__ double sell_combine(const double (*red)[32], int w0, int lane) {
  double a = red[w0][lane];
#pragma unroll
  for (int t = 1; t < kSplit; ++t) a += red[w0 + t][lane];
  return a;
}
struct Sell {
  int32_t o0, wd;   // first slot and width of the thread's slice (0 past the last slice)
};
__device__ __forceinline__ Sell sell_slice(const int32_t* off, int64_t ns, int64_t r) {
  const int64_t sl = r >> 5;
  Sell q{0, 0};
  if (sl < ns) {
    q.o0 = off[sl];
    q.wd = (off[sl + 1] - q.o0) >> 5;
  }
  return q;
}

// Complex shift s = s_r + i s_i: the right-hand side y = s M v_u + C v_u +
// M v_l of the operator is complex, y = (M w + C v_u) + i s_i (M v_u) with
// w = s_r v_u + v_l (k_scale); written interleaved (re, im) for the complex
// FB solve.
__global__ void __launch_bounds__(kSellBlock) k_spmv_op_c(
    const int32_t* off, int64_t ns, const int32_t* col, const double* Ms, const double* Cs,
    const double* vu, const double* w, double si, double* y, int64_t N) {
  pdl_trigger();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, sub = warp % kSplit;
  const int64_t r = ((int64_t)blockIdx.x * kSlicesPerBlock + warp / kSplit) * 32 + lane;
  const Sell q = sell_slice(off, ns, r);
  const int64_t e0 = q.o0 + lane;
  pdl_wait();
  double acc = 0.0, acm = 0.0;
#pragma unroll 2
  for (int k = sub; k < q.wd; k += kSplit) {
    const int64_t e = e0 + 32 * (int64_t)k;
    const int32_t c = col[e];
    const double m = Ms[e], u = vu[c];
    acc = fma(m, w[c], acc);
    acc = fma(Cs[e], u, acc);
    acm = fma(m, u, acm);
  }
  __shared__ double red[kSellBlock / 32][32];
  __shared__ double red2[kSellBlock / 32][32];
  red[warp][lane] = acc;
  red2[warp][lane] = acm;
  __syncthreads();
  if (sub == 0 && r < N) {
    y[2 * r] = sell_combine(red, warp, lane);
    y[2 * r + 1] = si * sell_combine(red2, warp, lane);
  }
}

// y_i = sum_q M_iq w_q + C_iq vu_q with w = s vu + vl (formed by k_scale when
// the basis vector was normalised): the fused s M v_u + C v_u + M v_l
__global__ void __launch_bounds__(kSellBlock) k_spmv_op(
    const int32_t* off, int64_t ns, const int32_t* col, const double* Ms, const double* Cs,
    const double* vu, const double* w, double* y, int64_t N) {
  pdl_trigger();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, sub = warp % kSplit;
  const int64_t r = ((int64_t)blockIdx.x * kSlicesPerBlock + warp / kSplit) * 32 + lane;
  // the pattern and the values are fixed before the chain starts (the first
  // step's share is loaded before the wait for the previous kernels); the
  // vectors are not
  const Sell q = sell_slice(off, ns, r);
  const int64_t e0 = q.o0 + lane;
  int32_t c[kSellUnroll];
  double mv[kSellUnroll], cv[kSellUnroll];
  auto load_step = [&](int k) {
#pragma unroll
    for (int t = 0; t < kSellUnroll; ++t) {
      const int64_t e = e0 + 32 * (int64_t)max(0, min(k + t * kSplit, q.wd - 1));
      c[t] = col[e];
      mv[t] = Ms[e];
      cv[t] = Cs[e];
    }
  };
  if (sub < q.wd) load_step(sub);
  pdl_wait();
  // kSellUnroll slots per step, every load of a step issued before its
  // products, so that the column-index loads and then the gathers overlap
  double acc = 0.0;
  for (int k = sub; k < q.wd; k += kSellUnroll * kSplit) {
    double wv[kSellUnroll], uv[kSellUnroll];
    if (k != sub) load_step(k);
#pragma unroll
    for (int t = 0; t < kSellUnroll; ++t) {
      wv[t] = w[c[t]];
      uv[t] = vu[c[t]];
    }
#pragma unroll
    for (int t = 0; t < kSellUnroll; ++t)
      if (k + t * kSplit < q.wd) {
        acc = fma(mv[t], wv[t], acc);
        acc = fma(cv[t], uv[t], acc);
      }
  }
  __shared__ double red[kSellBlock / 32][32];
  red[warp][lane] = acc;
  __syncthreads();
  if (sub == 0 && r < N) y[r] = sell_combine(red, warp, lane);
}

// h[c] = sum_i B(i, c) x(i) over the 2 Np rows of [V_u; W] (B-images of the
// basis vectors), x(i) = xa[i] (i < Np) or xb[i - Np]; then H[c, j] += h[c],
// for all ncol <= 96 columns in one launch.  The basis is streamed through
// shared memory by TMA: tiles of 128 rows x ncol columns rounded up to 8
// (boxes of 128 x 8), two stages, the next tile's copy in flight while the
// current one is used.  Warp w takes rows 32 (w mod 4) .. +31 of a tile and
// columns 32 (w / 4) .. +31; each lane keeps up to 32 column sums for its
// rows (only the loaded 8-column groups are accumulated, so that the FP64
// work follows ncol), reduced over the warp by a butterfly transpose once at
// the end; then the block's warps and the blocks are summed in a fixed order
// (last block to finish).  One block per SM.
constexpr int kTileRows = 128;
constexpr int kDotsCols = 96;    // columns per launch (the largest Krylov dimension)
constexpr int kDotsThreads = 384;
constexpr int kBoxCols = 8;
constexpr int kDotsGroups = 8;   // first stage of the cross-block sum
constexpr int kFbTimeEvery = 8;  // FB solves timed with CUDA events: one in eight
static_assert(kDotsCols >= kMaxKrylov, "one launch covers every basis column");
constexpr uint32_t kTmaWaitLimit = 1u << 22;

size_t dots_tma_smem() { return sizeof(double) * 2 * kDotsCols * kTileRows + 64; }

// acc[q] += tile[q * 128] * x for q < 8 G (G warp-uniform, 1..4)
template <int G>
__device__ __forceinline__ void dots_acc(double (&acc)[32], const double* tile, double x) {
#pragma unroll
  for (int q = 0; q < 8 * G; ++q) acc[q] = fma(tile[q * kTileRows], x, acc[q]);
}

__global__ void __launch_bounds__(kDotsThreads, 1)
    k_dots_tma(const __grid_constant__ CUtensorMap tV, int ncol, const double* xa,
               const double* xb, int64_t Np, double* part, unsigned* counter, double* h, double* H,
               int ldh, int j, DevStatus* st) {
  extern __shared__ __align__(1024) double dsm[];
  double* stage0 = dsm;
  double* stage1 = dsm + kDotsCols * kTileRows;
  // full[s]: the tile's copy landed (one arrival plus the bytes);
  // empty[s]: every warp has finished reading the stage (one arrival each)
  uint64_t* full = reinterpret_cast<uint64_t*>(dsm + 2 * kDotsCols * kTileRows);
  uint64_t* empty = full + 2;
  __shared__ double red[kDotsThreads / 32][32];
  __shared__ bool last;
  __shared__ volatile int abort_flag;
  const int64_t rows = 2 * Np;
  const int ntile = (int)((rows + kTileRows - 1) / kTileRows);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rs = (warp & 3) * 32, cg = warp >> 2;
  const int nbox = (ncol + kBoxCols - 1) / kBoxCols;
  // this warp's loaded 8-column groups (0..4)
  const int g = min(4, max(0, nbox - 4 * cg));
  const uint32_t bytes = (uint32_t)(nbox * kBoxCols * kTileRows * sizeof(double));
  pdl_trigger();
  if (threadIdx.x == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    mbar_init(&empty[0], kDotsThreads / 32);
    mbar_init(&empty[1], kDotsThreads / 32);
    abort_flag = 0;
    mbar_fence_init();
  }
  __syncthreads();
  // tile t covers rows t*128.. of [V_u; W]: V rows 0..Np-1, then 2Np..3Np-1
  auto vrow = [Np](int t) { const int64_t r = (int64_t)t * kTileRows; return (int)(r < Np ? r : r + Np); };
  // producer (thread 0): the block's first two tiles now, then each stage
  // again once every warp has released it.  The boxes of basis columns
  // 0..j-1 (normalised in earlier steps) are issued before the wait for the
  // previous kernels; the box holding column j (normalised at the end of
  // the previous step) and the columns past it after the wait.
  const int nb_early = min(nbox, j / kBoxCols);
  int issued[2] = {-1, -1};   // last iteration whose copy went to each stage
  if (threadIdx.x == 0)
    for (int st2 = 0; st2 < 2; ++st2) {
      const int t = (int)blockIdx.x + st2 * (int)gridDim.x;
      if (t < ntile) {
        double* dst = st2 ? stage1 : stage0;
        mbar_expect_tx(&full[st2], bytes);
        for (int b = 0; b < nb_early; ++b)
          tma_load_2d(dst + b * kBoxCols * kTileRows, &tV, vrow(t), kBoxCols * b, &full[st2]);
        issued[st2] = st2;
      }
    }
  pdl_wait();
  if (threadIdx.x == 0)
    for (int st2 = 0; st2 < 2; ++st2) {
      const int t = (int)blockIdx.x + st2 * (int)gridDim.x;
      if (t < ntile) {
        double* dst = st2 ? stage1 : stage0;
        for (int b = nb_early; b < nbox; ++b)
          tma_load_2d(dst + b * kBoxCols * kTileRows, &tV, vrow(t), kBoxCols * b, &full[st2]);
      }
    }
  double acc[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) acc[q] = 0.0;
  // this lane's entry of x for tile t (the next tile's load is issued a tile
  // ahead, so that its latency overlaps the current tile's products)
  auto xval = [&](int t) -> double {
    const int64_t i = (int64_t)t * kTileRows + rs + lane;
    return t < ntile ? (i < Np ? xa[i] : (i < rows ? xb[i - Np] : 0.0)) : 0.0;
  };
  double x = xval(blockIdx.x);
  int it = 0;
  for (int t = blockIdx.x; t < ntile; t += gridDim.x, ++it) {
    const int s = it & 1;
    const double* cur = s ? stage1 : stage0;
    const double xn = xval(t + (int)gridDim.x);
    const bool ok = __all_sync(0xffffffffu, mbar_wait(&full[s], (uint32_t)((it >> 1) & 1), kTmaWaitLimit));
    if (!ok) abort_flag = 1;
    if (abort_flag) break;
    const double* tile = cur + cg * 32 * kTileRows + rs + lane;   // column q at tile[q * 128]
    if (g == 4) dots_acc<4>(acc, tile, x);
    else if (g == 3) dots_acc<3>(acc, tile, x);
    else if (g == 2) dots_acc<2>(acc, tile, x);
    else if (g == 1) dots_acc<1>(acc, tile, x);
    x = xn;
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
    if (threadIdx.x == 0) {
      const int tn = t + 2 * (int)gridDim.x;
      if (tn < ntile) {
        if (!mbar_wait(&empty[s], (uint32_t)((it >> 1) & 1), kTmaWaitLimit)) {
          abort_flag = 1;
        } else {
          double* dst = s ? stage1 : stage0;
          mbar_expect_tx(&full[s], bytes);
          for (int b = 0; b < nbox; ++b)
            tma_load_2d(dst + b * kBoxCols * kTileRows, &tV, vrow(tn), kBoxCols * b, &full[s]);
          issued[s] = it + 2;
        }
      }
    }
  }
  __syncthreads();
  if (abort_flag) {
    if (threadIdx.x == 0) {
      atomicExch(&st->internal, 3);
      // let the copies still in flight into this block's shared memory land
      for (int st2 = 0; st2 < 2; ++st2)
        if (issued[st2] >= 0)
          mbar_wait(&full[st2], (uint32_t)((issued[st2] >> 1) & 1), kTmaWaitLimit);
    }
    __syncthreads();
    return;
  }
  // lane l <- the warp's sum for column 32 cg + l
  if (g > 0) {
#pragma unroll
    for (int o = 16, len = 32; o > 0; o >>= 1, len >>= 1) {
      bool up = (lane & o) != 0;
#pragma unroll
      for (int q = 0; q < len / 2; ++q) {
        double send = up ? acc[q] : acc[q + len / 2];
        double keep = up ? acc[q + len / 2] : acc[q];
        acc[q] = keep + __shfl_xor_sync(0xffffffffu, send, o);
      }
    }
  }
  red[warp][lane] = acc[0];
  __syncthreads();
  if (threadIdx.x < ncol) {
    const int cgr = threadIdx.x >> 5, l = threadIdx.x & 31;
    double sm = (red[4 * cgr][l] + red[4 * cgr + 1][l]) + (red[4 * cgr + 2][l] + red[4 * cgr + 3][l]);
    part[blockIdx.x * kDotsCols + threadIdx.x] = sm;
  }
  // Blocks sum in two stages, each in a fixed order: the last block of each
  // of ng groups (blocks g, g + ng, ...) adds its group's
  // partial sums, and the last group to finish adds the group sums.  Every
  // FP64 addition costs a 64-cycle issue slot, so one block summing all
  // gridDim x ncol partials (the tail of the launch) took several times as
  // long as the two short stages.
  const int ng = min(kDotsGroups, (int)gridDim.x);
  const int grp = (int)blockIdx.x % ng;
  const int gsize = ((int)gridDim.x - grp + ng - 1) / ng;
  double* gpart = part + (int64_t)gridDim.x * kDotsCols;   // kDotsGroups x 96 group sums
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(counter + 1 + grp, 1u) == (unsigned)gsize - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  // 384 threads: column c = tid mod 96, quarter = tid / 96 sums every fourth
  // block of the group (L2 loads; fixed order)
  const int c = threadIdx.x % kDotsCols, qtr = threadIdx.x / kDotsCols;
  double* red2 = &red[0][0];    // 4 x 96
  {
    double sm = 0.0;
    if (c < ncol)
      for (int b = grp + ng * qtr; b < (int)gridDim.x; b += 4 * ng)
        sm += __ldcg(part + b * kDotsCols + c);
    red2[qtr * kDotsCols + c] = sm;
  }
  __syncthreads();
  if (threadIdx.x < ncol)
    gpart[grp * kDotsCols + threadIdx.x] =
        (red2[threadIdx.x] + red2[kDotsCols + threadIdx.x]) +
        (red2[2 * kDotsCols + threadIdx.x] + red2[3 * kDotsCols + threadIdx.x]);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    counter[1 + grp] = 0u;
    last = (atomicAdd(counter, 1u) == (unsigned)ng - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x < ncol) {
    double v = 0.0;
#pragma unroll
    for (int g2 = 0; g2 < ng; ++g2) v += __ldcg(gpart + g2 * kDotsCols + threadIdx.x);
    h[threadIdx.x] = v;
    H[threadIdx.x + (int64_t)ldh * j] += v;
  }
  if (threadIdx.x == 0) *counter = 0u;
}

// B-norm of z = [zu; zl]: sum zu^2 + zl . (M zl) with the SpMV fused (8 lanes
// per row); the last block sets nrm = sqrt(sum), H[j+1, j] = nrm (if H),
// scal = {1/nrm, nrm}.
// B-norm of z = [zu; zl]: sum zu^2 + zl . (M zl) with the SpMV fused (SELL,
// one thread per row), M zl kept as the basis vector's B-image; the last
// block sets nrm = sqrt(sum), H[j+1, j] = nrm (if H), scal = {1/nrm, nrm}.
__global__ void __launch_bounds__(kSellBlock) k_bnorm(
    const int32_t* off, int64_t ns, const int32_t* col, const double* Ms, const double* zu,
    const double* zl, double* wz, int64_t N, double* part, unsigned* counter, double* H, int ldh,
    int j, double* scal, double bscale) {
  pdl_trigger();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, sub = warp % kSplit;
  const int64_t r = ((int64_t)blockIdx.x * kSlicesPerBlock + warp / kSplit) * 32 + lane;
  const Sell q = sell_slice(off, ns, r);
  const int64_t e0 = q.o0 + lane;
  int32_t c[kSellUnroll];
  double mv[kSellUnroll];
  auto load_step = [&](int k) {
#pragma unroll
    for (int t = 0; t < kSellUnroll; ++t) {
      const int64_t e = e0 + 32 * (int64_t)max(0, min(k + t * kSplit, q.wd - 1));
      c[t] = col[e];
      mv[t] = Ms[e];
    }
  };
  if (sub < q.wd) load_step(sub);   // the pattern and M: fixed before the chain
  pdl_wait();
  double acc = 0.0;
  for (int k = sub; k < q.wd; k += kSellUnroll * kSplit) {   // as in k_spmv_op
    double zv[kSellUnroll];
    if (k != sub) load_step(k);
#pragma unroll
    for (int t = 0; t < kSellUnroll; ++t) zv[t] = zl[c[t]];
#pragma unroll
    for (int t = 0; t < kSellUnroll; ++t)
      if (k + t * kSplit < q.wd) acc = fma(mv[t], zv[t], acc);
  }
  __shared__ double red[kSellBlock / 32][32];
  __shared__ double bs[kSlicesPerBlock];
  __shared__ bool last;
  const int nw = kSellBlock / 32;
  red[warp][lane] = acc;
  __syncthreads();
  if (sub == 0) {
    double v = 0.0;
    if (r < N) {
      const double a = bscale * sell_combine(red, warp, lane);
      wz[r] = a;   // (bscale M z_l)_r, the B-image kept with the basis vector
      v = zl[r] * a + zu[r] * zu[r];
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) bs[warp / kSplit] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sm = 0.0;
    for (int b = 0; b < kSlicesPerBlock; ++b) sm += bs[b];
    part[blockIdx.x] = sm;
    __threadfence();
    last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // L2 loads, several in flight; fixed-order sums over the blocks
  double sm = 0.0;
#pragma unroll 4
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) sm += __ldcg(part + b);
  for (int o = 16; o > 0; o >>= 1) sm += __shfl_xor_sync(0xffffffffu, sm, o);
  if (lane == 0) red[0][warp] = sm;
  __syncthreads();
  if (warp == 0) {
    double tot = lane < nw ? red[0][lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if (lane == 0) {
      double nr = sqrt(tot);
      if (H) H[(j + 1) + (int64_t)ldh * j] = nr;
      scal[0] = 1.0 / nr;
      scal[1] = nr;
      *counter = 0u;
    }
  }
}

// z[i] -= sum_c V[i, c] h[c] over the 2 Np rows of column z (ld stride in V)
// One row per thread, sixteen basis loads in flight (measured 0.1 ms per
// eigensolve ahead of eight), eight partial sums.  Launched as exactly as
// many equal blocks as fit on the SMs at once (a single balanced wave; see
// the launch).
__global__ void __launch_bounds__(1024) k_update(const double* V, int64_t ld, int ncol,
                                                 const double* h, double* z, int64_t rows) {
  pdl_trigger();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const double* vr = V + (i < rows ? i : 0);
  // the first eight basis columns, when all of them precede the newest one
  // (column ncol - 1, normalised at the end of the previous step), are
  // loaded before the wait for the previous kernels
  const bool early = ncol > 8 && i < rows;
  double v0[8];
  if (early) {
#pragma unroll
    for (int t = 0; t < 8; ++t) v0[t] = vr[ld * t];
  }
  pdl_wait();
  __shared__ double hs[kMaxKrylov + 1];
  for (int t = threadIdx.x; t <= kMaxKrylov; t += blockDim.x) hs[t] = t < ncol ? h[t] : 0.0;
  __syncthreads();
  if (i >= rows) return;
  double a[8];
#pragma unroll
  for (int t = 0; t < 8; ++t) a[t] = 0.0;
  int c = 0;
  if (early) {
#pragma unroll
    for (int t = 0; t < 8; ++t) a[t] = fma(v0[t], hs[t], a[t]);
    c = 8;
  }
  for (; c + 16 <= ncol; c += 16) {
    double v[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) v[t] = vr[ld * (c + t)];
#pragma unroll
    for (int t = 0; t < 16; ++t) a[t & 7] = fma(v[t], hs[c + t], a[t & 7]);
  }
  for (; c + 8 <= ncol; c += 8) {
    double v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) v[t] = vr[ld * (c + t)];
#pragma unroll
    for (int t = 0; t < 8; ++t) a[t] = fma(v[t], hs[c + t], a[t]);
  }
  for (; c < ncol; ++c) a[0] = fma(vr[ld * c], hs[c], a[0]);
  z[i] -= ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
}

// H[lock:m, lock:m] <- its symmetric part (the undamped pencil's projected
// matrix is symmetric; its entries outside the tridiagonal band are rounding
// from the full reorthogonalisation), so that the Ritz step sees a
// symmetric active block.  The locked leading columns stay as they are: the
// Ritz step relies on their decoupling (zero entries below them).
__global__ void k_symmetrize(double* H, int ldh, int m, int lock) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < m * m; q += gridDim.x * blockDim.x) {
    const int i = q % m, j = q / m;
    if (i < j && i >= lock) {
      const double v = 0.5 * (H[i + (int64_t)ldh * j] + H[j + (int64_t)ldh * i]);
      H[i + (int64_t)ldh * j] = v;
      H[j + (int64_t)ldh * i] = v;
    }
  }
}

// z *= 1 / ||z||_B over its 3 Np rows (v_u, v_l and the B-image M v_l);
// also w = s z_u + c z_l (rows < Np) for the next operator product (c = 1,
// or the scaling factor of the scaled pencil)
__global__ void k_scale(double* z, const double* scal, int64_t Np, double s, double c, double* w) {
  pdl_trigger();
  pdl_wait();
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < Np) {
    const double f = scal[0];
    const double u = z[i] * f, l = z[Np + i] * f;
    z[i] = u;
    z[Np + i] = l;
    z[2 * Np + i] *= f;
    w[i] = s * u + c * l;
  }
}

// out[i, t] = sum_{c < m} V[i, c] Q[c, t] (restart / basis change); each
// thread owns one row and 16 output columns t0 .. t0+15 (blockIdx.y).
__global__ void k_basis_gemm(const double* V, int64_t ld, int m, const double* Q, int k,
                             double* out, int64_t rows, int lo) {
  extern __shared__ double qs[];
  int t0 = lo + blockIdx.y * 16;
  int nt = min(16, k - t0);
  for (int i = threadIdx.x; i < m * 16; i += blockDim.x) {
    int c = i % m, q = i / m;
    qs[i] = q < nt ? Q[c + m * (t0 + q)] : 0.0;
  }
  __syncthreads();
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= rows) return;
  double acc[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = 0.0;
  const double* vr = V + i;
  for (int c = lo; c < m; ++c) {
    double v = vr[ld * c];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] += v * qs[c + m * q];
  }
  for (int q = 0; q < nt; ++q) out[i + ld * (t0 + q)] = acc[q];
}

// start vector in the original order: splitmix64(seed + i) / 2^64 - 0.5
__global__ void k_start_vector(uint64_t seed, double* v, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t z = seed + (uint64_t)i + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  v[i] = (double)(z >> 11) * 0x1.0p-53 - 0.5;
}

// V_u(:,0)[j] = v1[perm[j]], V_l(:,0)[j] = v1[N + perm[j]]
__global__ void k_load_start(const double* v1, const int32_t* perm, double* V0, int64_t N,
                             int64_t Np) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= N) return;
  int32_t o = perm[j];
  V0[j] = v1[o];
  V0[Np + j] = v1[N + o];
}

// Xn[i, t] = sum_c V_u[i, c] Y[c, t] (complex Y), scattered to the original order
__global__ void k_eigvec(const double* V, int64_t ld, int m, const double* Y, int neig,
                         const int32_t* perm, double* X, int64_t N) {
  extern __shared__ double ys[];
  for (int i = threadIdx.x; i < 2 * m * neig; i += blockDim.x) ys[i] = Y[i];
  __syncthreads();
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  int64_t o = perm[i];
  for (int t = 0; t < neig; ++t) {
    double ar = 0.0, ai = 0.0;
    for (int c = 0; c < m; ++c) {
      double v = V[i + ld * c];
      ar += v * ys[2 * (c + m * t)];
      ai += v * ys[2 * (c + m * t) + 1];
    }
    X[2 * (o + N * t)] = ar;
    X[2 * (o + N * t) + 1] = ai;
  }
}

// per column: ||x||^2 and the largest |x_i| (lowest index on ties)
__global__ void k_colstats(const double* X, int64_t N, double* stats) {
  int t = blockIdx.x;
  const double* x = X + 2 * N * t;
  double s = 0.0, best = -1.0;
  int64_t bi = 0;
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
    double a2 = x[2 * i] * x[2 * i] + x[2 * i + 1] * x[2 * i + 1];
    s += a2;
    if (a2 > best) { best = a2; bi = i; }
  }
  __shared__ double ss[1024], sb[1024];
  __shared__ int64_t si[1024];
  ss[threadIdx.x] = s;
  sb[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      ss[threadIdx.x] += ss[threadIdx.x + w];
      double b2 = sb[threadIdx.x + w];
      int64_t i2 = si[threadIdx.x + w];
      if (b2 > sb[threadIdx.x] || (b2 == sb[threadIdx.x] && i2 < si[threadIdx.x])) {
        sb[threadIdx.x] = b2;
        si[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    stats[4 * t] = ss[0];
    stats[4 * t + 1] = (double)si[0];
    stats[4 * t + 2] = x[2 * si[0]];
    stats[4 * t + 3] = x[2 * si[0] + 1];
  }
}

// x <- x * conj(x_imax) / (|x_imax| ||x||)
__global__ void k_colnormalise(double* X, int64_t N, const double* stats) {
  int t = blockIdx.y;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  double* x = X + 2 * N * t;
  double pr = stats[4 * t + 2], pi = stats[4 * t + 3];
  double pa = hypot(pr, pi);
  double sc = 1.0 / (pa * sqrt(stats[4 * t]));
  // (a + ib)(pr - i pi)
  double a = x[2 * i], b = x[2 * i + 1];
  double nr = (a * pr + b * pi) * sc, ni = (b * pr - a * pi) * sc;
  x[2 * i] = nr;
  x[2 * i + 1] = ni;
}

// partial sums of ||K x + l C x + l^2 M x||^2 and ||x||^2 for column t
__global__ void k_qres(const int32_t* rowptr, const int32_t* col, const double* K, const double* M,
                       const double* C, const double* X, const double* lam, int64_t N,
                       double* part, double cfac) {
  int t = blockIdx.y;
  const double* x = X + 2 * N * t;
  double lr = lam[2 * t], li = lam[2 * t + 1];
  double l2r = lr * lr - li * li, l2i = 2 * lr * li;
  double s = 0.0, sx = 0.0;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < N;
       r += (int64_t)gridDim.x * blockDim.x) {
    double kr = 0, ki = 0, cr = 0, ci = 0, mr = 0, mi = 0;
    for (int32_t q = rowptr[r]; q < rowptr[r + 1]; ++q) {
      double xr = x[2 * col[q]], xi = x[2 * col[q] + 1];
      kr += K[q] * xr; ki += K[q] * xi;
      cr += C[q] * xr; ci += C[q] * xi;
      mr += M[q] * xr; mi += M[q] * xi;
    }
    double rr = kr + cfac * (lr * cr - li * ci) + (l2r * mr - l2i * mi);
    double ri = ki + cfac * (lr * ci + li * cr) + (l2r * mi + l2i * mr);
    s += rr * rr + ri * ri;
    sx += x[2 * r] * x[2 * r] + x[2 * r + 1] * x[2 * r + 1];
  }
  __shared__ double a[256], b[256];
  a[threadIdx.x] = s;
  b[threadIdx.x] = sx;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) { a[threadIdx.x] += a[threadIdx.x + w]; b[threadIdx.x] += b[threadIdx.x + w]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * (blockIdx.x + gridDim.x * t)] = a[0];
    part[2 * (blockIdx.x + gridDim.x * t) + 1] = b[0];
  }
}

__global__ void k_eta(const double* part, int nblk, const double* lam, double nK, double nM,
                      double nC, double* eta, int neig) {
  int t = threadIdx.x;
  if (t >= neig) return;
  double s = 0.0, sx = 0.0;
  for (int b = 0; b < nblk; ++b) {
    s += part[2 * (b + nblk * t)];
    sx += part[2 * (b + nblk * t) + 1];
  }
  double al = hypot(lam[2 * t], lam[2 * t + 1]);
  eta[t] = sqrt(s) / ((al * al * nM + al * nC + nK) * sqrt(sx));
}

// ---- damping sensitivity ----
// partial sums of x^T (2 l M + C) x (unconjugated) for column t
__global__ void k_gden(const int32_t* rowptr, const int32_t* col, const double* M, const double* C,
                       const double* X, const double* lam, int64_t N, double* part) {
  int t = blockIdx.y;
  const double* x = X + 2 * N * t;
  double lr = lam[2 * t], li = lam[2 * t + 1];
  double sr = 0.0, si = 0.0;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < N;
       r += (int64_t)gridDim.x * blockDim.x) {
    double mr = 0, mi = 0, cr = 0, ci = 0;
    for (int32_t q = rowptr[r]; q < rowptr[r + 1]; ++q) {
      double xr = x[2 * col[q]], xi = x[2 * col[q] + 1];
      mr += M[q] * xr; mi += M[q] * xi;
      cr += C[q] * xr; ci += C[q] * xi;
    }
    // w = 2 l (Mx) + Cx ; accumulate x_r * w
    double wr = 2 * (lr * mr - li * mi) + cr, wi = 2 * (lr * mi + li * mr) + ci;
    double xr = x[2 * r], xi = x[2 * r + 1];
    sr += xr * wr - xi * wi;
    si += xr * wi + xi * wr;
  }
  __shared__ double a[256], b[256];
  a[threadIdx.x] = sr;
  b[threadIdx.x] = si;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) { a[threadIdx.x] += a[threadIdx.x + w]; b[threadIdx.x] += b[threadIdx.x + w]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * (blockIdx.x + gridDim.x * t)] = a[0];
    part[2 * (blockIdx.x + gridDim.x * t) + 1] = b[0];
  }
}

__global__ void k_gden_final(const double* part, int nblk, int neig, double* den) {
  int t = threadIdx.x;
  if (t >= neig) return;
  double sr = 0, si = 0;
  for (int b = 0; b < nblk; ++b) { sr += part[2 * (b + nblk * t)]; si += part[2 * (b + nblk * t) + 1]; }
  den[2 * t] = sr;
  den[2 * t + 1] = si;
}

// G[t, e] = -l_t q_{t,e} / den_t with q = x_e^T (mx (x) my) x_e over the
// element's (p+1)^2 functions (Dirichlet functions carry no DOF)
// k_grad for a fixed p + 1 = NP: the element form x_e^T (my (x) mx) x_e as
// sum_{b,d} my[b,d] (X^T (mx X))[b,d] (X the NP x NP block of x on the
// element, complex, unconjugated) in registers: 6 NP^3 FMAs instead of the
// NP^4 of the direct double sum.
template <int NP>
__global__ void __launch_bounds__(128) k_grad_p(const double* X, const double* lam,
                                                const double* den, const double* m1,
                                                const int* first_fn, int ne, int n1, int64_t N,
                                                int neig, double* G) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t ne2 = (int64_t)ne * ne;
  if (tid >= ne2 * neig) return;
  const int t = (int)(tid / ne2);
  const int64_t e = tid % ne2;
  const int ex = (int)(e % ne), ey = (int)(e / ne);
  const double* x = X + 2 * N * t;
  double xr[NP][NP], xi[NP][NP];
  const int fx = first_fn[ex] - 1, fy = first_fn[ey] - 1;
#pragma unroll
  for (int a = 0; a < NP; ++a)
#pragma unroll
    for (int b = 0; b < NP; ++b) {
      const int dx = fx + a, dy = fy + b;
      const bool in = dx >= 0 && dx < n1 && dy >= 0 && dy < n1;
      const int64_t d = in ? dx + (int64_t)n1 * dy : 0;
      xr[a][b] = in ? __ldg(x + 2 * d) : 0.0;
      xi[a][b] = in ? __ldg(x + 2 * d + 1) : 0.0;
    }
  const double* mx = m1 + (int64_t)ex * NP * NP;
  const double* my = m1 + (int64_t)ey * NP * NP;
  double qr = 0.0, qi = 0.0;
#pragma unroll
  for (int d = 0; d < NP; ++d) {
    // column d of T = mx X
    double tr[NP], ti[NP];
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      double sr = 0.0, si = 0.0;
#pragma unroll
      for (int c = 0; c < NP; ++c) {
        const double m = __ldg(mx + a * NP + c);
        sr = fma(m, xr[c][d], sr);
        si = fma(m, xi[c][d], si);
      }
      tr[a] = sr;
      ti[a] = si;
    }
#pragma unroll
    for (int b = 0; b < NP; ++b) {
      double wr = 0.0, wi = 0.0;   // W[b][d] = sum_a X[a][b] T[a][d]
#pragma unroll
      for (int a = 0; a < NP; ++a) {
        wr = fma(xr[a][b], tr[a], fma(-xi[a][b], ti[a], wr));
        wi = fma(xr[a][b], ti[a], fma(xi[a][b], tr[a], wi));
      }
      const double mbd = __ldg(my + b * NP + d);
      qr = fma(mbd, wr, qr);
      qi = fma(mbd, wi, qi);
    }
  }
  const double lr = lam[2 * t], li = lam[2 * t + 1];
  const double nr = -(lr * qr - li * qi), ni = -(lr * qi + li * qr);
  const double dr = den[2 * t], di = den[2 * t + 1];
  const double dd = dr * dr + di * di;
  G[2 * (e + ne2 * t)] = (nr * dr + ni * di) / dd;
  G[2 * (e + ne2 * t) + 1] = (ni * dr - nr * di) / dd;
}

__global__ void k_grad(const double* X, const double* lam, const double* den, const double* m1,
                       const int* first_fn, int ne, int p, int n1, int64_t N, int neig,
                       double* G) {
  int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t ne2 = (int64_t)ne * ne;
  if (tid >= ne2 * neig) return;
  int t = tid / ne2;
  int64_t e = tid % ne2;
  int ex = e % ne, ey = e / ne;
  int np1 = p + 1;
  const double* x = X + 2 * N * t;
  double xr[kMaxP + 1][kMaxP + 1], xi[kMaxP + 1][kMaxP + 1];
  for (int a = 0; a < np1; ++a)
    for (int b = 0; b < np1; ++b) {
      int dx = first_fn[ex] + a - 1, dy = first_fn[ey] + b - 1;
      if (dx >= 0 && dx < n1 && dy >= 0 && dy < n1) {
        int64_t d = dx + (int64_t)n1 * dy;
        xr[a][b] = x[2 * d];
        xi[a][b] = x[2 * d + 1];
      } else {
        xr[a][b] = 0.0;
        xi[a][b] = 0.0;
      }
    }
  const double* mx = m1 + (int64_t)ex * np1 * np1;
  const double* my = m1 + (int64_t)ey * np1 * np1;
  double qr = 0.0, qi = 0.0;
  for (int b = 0; b < np1; ++b)
    for (int d = 0; d < np1; ++d) {
      // W[b][d] = sum_{a,c} x[a][b] mx[a][c] x[c][d]
      double wr = 0.0, wi = 0.0;
      for (int a = 0; a < np1; ++a) {
        double tr = 0.0, ti = 0.0;
        for (int c = 0; c < np1; ++c) {
          double mac = mx[a * np1 + c];
          tr += mac * xr[c][d];
          ti += mac * xi[c][d];
        }
        wr += xr[a][b] * tr - xi[a][b] * ti;
        wi += xr[a][b] * ti + xi[a][b] * tr;
      }
      double mbd = my[b * np1 + d];
      qr += mbd * wr;
      qi += mbd * wi;
    }
  // g = -l q / den
  double lr = lam[2 * t], li = lam[2 * t + 1];
  double nr = -(lr * qr - li * qi), ni = -(lr * qi + li * qr);
  double dr = den[2 * t], di = den[2 * t + 1];
  double dd = dr * dr + di * di;
  G[2 * (e + ne2 * t)] = (nr * dr + ni * di) / dd;
  G[2 * (e + ne2 * t) + 1] = (ni * dr - nr * di) / dd;
}

// basis layout: rows per half (a multiple of the TMA tile) and column stride
int64_t basis_np(int64_t N) { return (N + kTileRows - 1) / kTileRows * kTileRows; }
int64_t basis_ld(int64_t N) { return 3 * basis_np(N); }

struct Work {
  Problem& P;
  int m;
  int64_t N, Np, ld;
  int nblk;
  cudaStream_t s;
  double sigma;
  double vscale = 1.0;   // scaling factor of the scaled pencil (1: unscaled)
  // FB outputs r_u = -fb_uscale x, r_l = -fb_sigma x + v_u: the QEP operator
  // (sigma, vscale), or r_l = x, r_u = 0 for the undamped pencil (-1, 0)
  double fb_sigma = 0.0, fb_uscale = 1.0;
  double shift_i = 0.0;   // imaginary part of a complex shift (0: real operator)
  int64_t n_apply = 0, n_spmv = 0, n_vv = 0;
  // FB timing: event pairs around every kFbTimeEvery-th FB solve (an event
  // between two kernels ends the programmatic overlap of their launches:
  // events around every solve cost 0.75 ms per eigensolve of the 256^2
  // workload); fb_ms sums the timed solves, fb_timed counts them
  std::vector<cudaEvent_t> ev;
  int ev_used = 0;
  double fb_ms = 0.0;
  int64_t fb_timed = 0;
  cudaEvent_t rz[2] = {nullptr, nullptr};   // around each Ritz step
  double ritz_ms = 0.0;
  CUtensorMap tV{};  // the Krylov basis V for the TMA-fed kernels
  int nsm = 0;       // SMs of the device (one TMA block each)
  int upd_threads = 256;   // k_update block: equal blocks, as many per SM as fit
  ~Work() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    for (cudaEvent_t e : rz)
      if (e) cudaEventDestroy(e);
  }
  void fb_events(int count) {
    while ((int)ev.size() < 2 * count) {
      cudaEvent_t e;
      RQ_CUDA(cudaEventCreate(&e));
      ev.push_back(e);
    }
  }
  // after a stream synchronisation: add the elapsed FB time of this cycle
  void fb_collect() {
    for (int i = 0; i + 1 < ev_used; i += 2) {
      float ms = 0.f;
      RQ_CUDA(cudaEventElapsedTime(&ms, ev[i], ev[i + 1]));
      fb_ms += ms;
      ++fb_timed;
    }
    ev_used = 0;
  }

  double* col(int c) { return P.V.p + ld * c; }

  void dots(int j, const double* xa, const double* xb) {
    launch_pdl(k_dots_tma, dim3(nsm), dim3(kDotsThreads), dots_tma_smem(), s, tV, j + 1, xa, xb, Np,
               P.part.p, P.counter.p + 4, P.hvec.p, P.H.p, m + 1, j, P.status.p);
    ++P.launches;
  }
  // B-norm of column c -> H[c, c-1] (if setH) and V[:, c] normalised
  void normalise(int c, bool setH) {
    double* z = col(c);
    const int64_t ns = (N + 31) / 32;
    launch_pdl(k_bnorm, dim3((unsigned)((ns + kSlicesPerBlock - 1) / kSlicesPerBlock)),
               dim3(kSellBlock), 0, s, P.sell_off.p, ns,
               P.sell_col.p, P.sell_M.p, z,
               (const double*)(z + Np), z + 2 * Np, N, P.part.p, P.counter.p + 1,
               setH ? P.H.p : nullptr, m + 1, c - 1, P.scal.p, vscale * vscale);
    ++n_spmv;
    P.launches += 2;
    launch_pdl(k_scale, dim3((unsigned)((Np + 255) / 256)), dim3(256), 0, s, z,
               (const double*)P.scal.p, Np, sigma, vscale, P.wop.p);
    n_vv += 2;
  }
  void step(int j) {
    double* v = col(j);
    double* r = col(j + 1);
    const int64_t ns = (N + 31) / 32;
    const bool timed = n_apply % kFbTimeEvery == 0;
    if (shift_i != 0.0) {
      // complex shift: Re((A - s B)^{-1} B v) through the complex factor
      launch_pdl(k_spmv_op_c, dim3((unsigned)((ns + kSlicesPerBlock - 1) / kSlicesPerBlock)),
                 dim3(kSellBlock), 0, s, P.sell_off.p, ns, P.sell_col.p, P.sell_M.p, P.sell_C.p,
                 (const double*)v, (const double*)P.wop.p, shift_i, (double*)P.cx.y.p, N);
      n_spmv += 4;
      if (timed) RQ_CUDA(cudaEventRecord(ev[ev_used++], s));
      launch_fb_complex(P, P.cx.y.p, sigma, shift_i, v, r, r + Np);
      if (timed) RQ_CUDA(cudaEventRecord(ev[ev_used++], s));
    } else {
      launch_pdl(k_spmv_op, dim3((unsigned)((ns + kSlicesPerBlock - 1) / kSlicesPerBlock)),
                 dim3(kSellBlock), 0, s, P.sell_off.p,
                 ns, P.sell_col.p, P.sell_M.p, P.sell_C.p, (const double*)v, (const double*)P.wop.p,
                 P.yop.p, N);
      n_spmv += 3;
      if (timed) RQ_CUDA(cudaEventRecord(ev[ev_used++], s));
      launch_fb(P, P.yop.p, fb_sigma, v, r, r + Np, fb_uscale);
      if (timed) RQ_CUDA(cudaEventRecord(ev[ev_used++], s));
    }
    ++n_apply;
    for (int pass = 0; pass < 2; ++pass) {
      dots(j, r, r + Np);   // V_u^T r_u + W^T r_l
      launch_pdl(k_update, dim3((unsigned)((2 * Np + upd_threads - 1) / upd_threads)),
                 dim3((unsigned)upd_threads), 0, s, (const double*)P.V.p, ld, j + 1,
                 (const double*)P.hvec.p, r, 2 * Np);
      ++P.launches;
      n_vv += 4 * (j + 1);
    }
    normalise(j + 1, true);
  }
};

// Krylov-Schur iteration of the shift-and-invert operator until the ncand
// wanted Ritz pairs converge (or max_restarts): leaves the basis in P.V, the
// eigenvectors of H for the candidates in P.Y and the candidates in P.cand.
void krylov_schur(Problem& P, const EigsParams& E, const double* v1) {
  Plan& L = P.plan;
  cudaStream_t s = P.stream;
  const int m = E.m, max_restarts = E.max_restarts;
  const int nks = E.ncand;          // pairs converged around the shift
  const double sigma = E.shift, tol = E.tol;
  const uint64_t seed = E.seed;
  Work W{P, m, L.N, 0, 0, 0, s, sigma};
  W.vscale = E.vscale;
  W.fb_sigma = E.gep ? -1.0 : sigma;
  W.fb_uscale = E.gep ? 0.0 : E.vscale;
  if (E.gep) W.sigma = 0.0;   // w = 0 * v_u + v_l: the operator input is v_l alone
  W.shift_i = E.cplx ? E.shift_i : 0.0;
  W.fb_events(m + 1);
  RQ_CUDA(cudaEventCreate(&W.rz[0]));
  RQ_CUDA(cudaEventCreate(&W.rz[1]));
  W.Np = basis_np(L.N);
  W.ld = basis_ld(L.N);
  W.nblk = 2 * P.nsm;
  int64_t ld = W.ld, Np = W.Np, N = L.N;
  P.V.alloc(ld * (m + 1));
  make_tmap_f64(&W.tV, P.V.p, (uint64_t)ld, (uint64_t)(m + 1), (uint64_t)ld, kTileRows, kBoxCols);
  {
    int dev = 0;
    RQ_CUDA(cudaGetDevice(&dev));
    RQ_CUDA(cudaDeviceGetAttribute(&W.nsm, cudaDevAttrMultiProcessorCount, dev));
    smem_at_least((const void*)k_dots_tma, dots_tma_smem());
    // rows of the update split into bps * nsm blocks of whole warps (<= 1024),
    // bps the number of such blocks that fit on an SM: when more fit than the
    // grid gives each SM, the SMs that free up first (the launch overlaps the
    // previous kernel's tail) take the extra blocks and the others idle.  A
    // 32-register build of this kernel let a third 544-thread block onto an
    // SM and took 25-38% longer in the eigensolve than the 48-register one.
    for (int bps = 2;;) {
      const int64_t per = (2 * W.Np + bps * W.nsm - 1) / (bps * (int64_t)W.nsm);
      W.upd_threads = (int)std::min<int64_t>(1024, std::max<int64_t>(32, (per + 31) / 32 * 32));
      int occ = 0;
      RQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_update, W.upd_threads, 0));
      if (occ <= bps || bps >= 32) break;
      bps = occ;
    }
  }
  P.Vtmp.alloc(ld * m);
  P.H.alloc((m + 1) * m);
  P.part.alloc(64 * (size_t)std::max(W.nblk, 4 * 1024) + (size_t)(L.N * 8 + 255) / 256);
  P.counter.alloc(16);
  RQ_CUDA(cudaMemsetAsync(P.counter.p, 0, 16 * sizeof(unsigned), s));
  P.hvec.alloc(kMaxKrylov + 1);
  P.yop.alloc(Np);
  P.wop.alloc(Np);
  P.scal.alloc(4);
  P.Y.alloc(2 * (size_t)m * kMaxKrylov);
  P.ritz.alloc(1);
  DBuf<double> Hn, Qb, v1buf;
  Hn.alloc((m + 1) * m);
  Qb.alloc((size_t)m * m);
  RQ_CUDA(cudaMemsetAsync(P.V.p, 0, sizeof(double) * ld * (m + 1), s));
  RQ_CUDA(cudaMemsetAsync(P.Vtmp.p, 0, sizeof(double) * ld * m, s));
  RQ_CUDA(cudaMemsetAsync(P.H.p, 0, sizeof(double) * (m + 1) * m, s));

  const double* start = v1;
  if (!start) {
    v1buf.alloc(2 * N);
    k_start_vector<<<(unsigned)((2 * N + 255) / 256), 256, 0, s>>>(seed, v1buf.p, 2 * N);
    RQ_CUDA(cudaGetLastError());
    start = v1buf.p;
  }
  k_load_start<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(start, P.perm.p, P.V.p, N, Np);
  RQ_CUDA(cudaGetLastError());
  if (E.gep)   // undamped pencil: the basis lives in the lower block
    RQ_CUDA(cudaMemsetAsync(P.V.p, 0, sizeof(double) * Np, s));
  W.normalise(0, false);

  // kept at a restart: the candidates plus two (measured: fewer operator
  // applications and Ritz steps than keeping half of the extra vectors)
  int kwant = std::min(nks + 2, std::max(nks, m - 2));
  int k = 0;
  int lock = 0;   // leading Schur columns locked (converged, decoupled)
  RitzOut h_out{};
  int restarts = 0;
  for (int q = 0; q < 6; ++q) P.info.ritz_phase_cycles[q] = 0.0;
  int64_t qr_sweeps = 0;
  for (int it = 0;; ++it) {
    for (int j = k; j < m; ++j) W.step(j);
    RQ_CUDA(cudaEventRecord(W.rz[0], s));
    // the last allowed cycle always finishes; the others finish when converged
    if (E.gep) {
      k_symmetrize<<<(unsigned)((m * m + 255) / 256), 256, 0, s>>>(P.H.p, m + 1, m, lock);
      RQ_CUDA(cudaGetLastError());
      ++P.launches;
    }
    // complex shift: the Ritz values theta of the real operator map to the
    // eigenvalues through a quadratic (eigs_run); the step reports 1 / theta
    launch_ritz(P.H.p, Hn.p, Qb.p, P.Y.p, P.ritz.p, m, nks, kwant, it >= max_restarts ? 1 : 2,
                lock, E.cplx ? 0.0 : sigma, tol, E.cplx ? 1.0 : E.vscale, s);
    RQ_CUDA(cudaEventRecord(W.rz[1], s));
    ++P.launches;
    RQ_CUDA(cudaMemcpyAsync(&h_out, P.ritz.p, sizeof(RitzOut), cudaMemcpyDeviceToHost, s));
    RQ_CUDA(cudaStreamSynchronize(s));
    W.fb_collect();
    {
      float ms = 0.f;
      RQ_CUDA(cudaEventElapsedTime(&ms, W.rz[0], W.rz[1]));
      W.ritz_ms += ms;
    }
    if (h_out.fail == 2)
      throw Error(RIGAQEP_ERR_TIMEOUT, "a bounded wait between the Ritz-step CTAs ran out");
    if (h_out.fail) throw Error(RIGAQEP_ERR_INTERNAL, "QR iteration on the projected matrix did not converge");
    qr_sweeps += h_out.sweeps;
    for (int q = 0; q < 6; ++q) P.info.ritz_phase_cycles[q] += (double)h_out.phase_cycles[q];
    if (h_out.finished) break;
    k = h_out.k;
    // the columns locked before this Ritz step are untouched by it: their
    // Schur vectors are unit vectors (Q[:lk, :lk] = I, Q[:lk, lk:] = 0), so
    // only V[:, lk:k] = V[:, lk:m] Q[lk:m, lk:k] is formed
    const int lk = lock;
    lock = h_out.n_lock;
    // V[:, :k] = V[:, :m] Q ; V[:, k] = V[:, m] ; H = Hnew
    size_t smem = sizeof(double) * (size_t)m * 16;
    if (k > lk) {
      dim3 gg((unsigned)((ld + 127) / 128), (unsigned)((k - lk + 15) / 16));
      k_basis_gemm<<<gg, 128, smem, s>>>(P.V.p, ld, m, Qb.p, k, P.Vtmp.p, ld, lk);
      RQ_CUDA(cudaGetLastError());
      ++P.launches;
      RQ_CUDA(cudaMemcpyAsync(P.V.p + ld * lk, P.Vtmp.p + ld * lk, sizeof(double) * ld * (k - lk),
                              cudaMemcpyDeviceToDevice, s));
    }
    RQ_CUDA(cudaMemcpyAsync(P.V.p + ld * k, P.V.p + ld * m, sizeof(double) * ld,
                            cudaMemcpyDeviceToDevice, s));
    RQ_CUDA(cudaMemcpyAsync(P.H.p, Hn.p, sizeof(double) * (m + 1) * m, cudaMemcpyDeviceToDevice, s));
    ++restarts;
  }
  P.cand = h_out;
  P.cand_E = E;
  P.cand_valid = v1 == nullptr;   // a seeded start vector can be reproduced
  P.info.n_apply = W.n_apply;
  P.info.n_restarts = restarts;
  P.info.n_spmv = W.n_spmv;
  P.info.n_vv = W.n_vv;
  P.info.n_qr_sweeps = qr_sweeps;
  // every solve runs the same kernels: the timed ones' mean times the count
  P.info.fb_ms = W.fb_timed > 0 ? W.fb_ms * (double)W.n_apply / (double)W.fb_timed : 0.0;
  P.info.ritz_ms = W.ritz_ms;
  P.info.reused_candidates = 0;
}

bool same_candidates(const EigsParams& a, const EigsParams& b) {
  return a.in_region && b.in_region && a.shift == b.shift && a.ncand == b.ncand && a.m == b.m &&
         a.max_restarts == b.max_restarts && a.tol == b.tol && a.seed == b.seed &&
         a.vscale == b.vscale;
}

}  // namespace

void make_tmap_f64(CUtensorMap* map, const double* base, uint64_t rows, uint64_t cols, uint64_t ld,
                   uint32_t box_rows, uint32_t box_cols) {
  using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                              CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                              CUtensorMapFloatOOBfill);
  static Encode encode = nullptr;
  static std::mutex mu;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!encode) {
      void* fn = nullptr;
      cudaDriverEntryPointQueryResult q;
      RQ_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                               cudaEnableDefault, &q));
      if (q != cudaDriverEntryPointSuccess || !fn)
        throw Error(RIGAQEP_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
      encode = (Encode)fn;
    }
  }
  cuuint64_t dims[2] = {rows, cols};
  cuuint64_t strides[1] = {ld * sizeof(double)};
  cuuint32_t box[2] = {box_rows, box_cols};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, (void*)base, dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error(RIGAQEP_ERR_CUDA, "cuTensorMapEncodeTiled failed");
}

// Complex shift s (Section 4.1.1 allows s in C): the Krylov iteration ran on
// the real operator R = Re((A - s B)^{-1} B) = ((A - s B)^{-1} + (A - conj(s)
// B)^{-1}) B / 2, whose eigenvalue for an eigenpair (lambda, z) of the pencil
// is psi = (1/(lambda - s) + 1/(lambda - conj s)) / 2 = (lambda - a) /
// ((lambda - s)(lambda - conj s)), a = Re s.  Each converged psi gives two
// candidate eigenvalues, the roots of psi l^2 - (2 a psi + 1) l + psi |s|^2 +
// a = 0; the eigenvector x = V_u y decides between them (the root with the
// smaller QEP backward error).  The neig eigenvalues nearest s are returned.
void finish_complex(Problem& P, const EigsParams& E, double* lambda, double* X, double* eta,
                    int* n_conv) {
  Plan& L = P.plan;
  cudaStream_t s = P.stream;
  const int m = E.m, nc = E.ncand, neig = E.neig;
  const int64_t N = L.N, ld = basis_ld(L.N);
  const RitzOut& h = P.cand;
  const std::complex<double> sh(E.shift, E.shift_i);
  const double a = E.shift, s2 = std::norm(sh);
  std::vector<double> r1(2 * (size_t)nc), r2(2 * (size_t)nc);
  for (int i = 0; i < nc; ++i) {
    const std::complex<double> psi = 1.0 / std::complex<double>(h.lam[2 * i], h.lam[2 * i + 1]);
    const std::complex<double> qa = psi, qb = -(2.0 * a * psi + 1.0), qc = psi * s2 + a;
    const std::complex<double> d = std::sqrt(qb * qb - 4.0 * qa * qc);
    const std::complex<double> x1 = (-qb + d) / (2.0 * qa), x2 = (-qb - d) / (2.0 * qa);
    r1[2 * i] = x1.real();
    r1[2 * i + 1] = x1.imag();
    r2[2 * i] = x2.real();
    r2[2 * i + 1] = x2.imag();
  }
  DBuf<double> Xa, l1, l2, e1, e2, stats;
  Xa.alloc(2 * (size_t)N * nc);
  {
    size_t smem = sizeof(double) * 2 * (size_t)m * nc;
    smem_at_least((const void*)k_eigvec, smem);
    k_eigvec<<<(unsigned)((N + 127) / 128), 128, smem, s>>>(P.V.p, ld, m, P.Y.p, nc, P.perm.p,
                                                           Xa.p, N);
    RQ_CUDA(cudaGetLastError());
  }
  stats.alloc(4 * (size_t)nc);
  k_colstats<<<nc, 1024, 0, s>>>(Xa.p, N, stats.p);
  RQ_CUDA(cudaGetLastError());
  k_colnormalise<<<dim3((unsigned)((N + 255) / 256), nc), 256, 0, s>>>(Xa.p, N, stats.p);
  RQ_CUDA(cudaGetLastError());
  l1.upload(r1, s);
  l2.upload(r2, s);
  e1.alloc(nc);
  e2.alloc(nc);
  const int qb = 2 * P.nsm;
  for (int pass = 0; pass < 2; ++pass) {
    k_qres<<<dim3(qb, nc), 256, 0, s>>>(P.rowptr.p, P.col.p, P.K.p, P.M.p, P.C.p, Xa.p,
                                       pass ? l2.p : l1.p, N, P.part.p, 1.0);
    RQ_CUDA(cudaGetLastError());
    k_eta<<<1, 128, 0, s>>>(P.part.p, qb, pass ? l2.p : l1.p, P.info.norm_K, P.info.norm_M,
                            P.info.norm_C, pass ? e2.p : e1.p, nc);
    RQ_CUDA(cudaGetLastError());
  }
  P.launches += 7;
  std::vector<double> h1(nc), h2(nc);
  RQ_CUDA(cudaMemcpyAsync(h1.data(), e1.p, sizeof(double) * nc, cudaMemcpyDeviceToHost, s));
  RQ_CUDA(cudaMemcpyAsync(h2.data(), e2.p, sizeof(double) * nc, cudaMemcpyDeviceToHost, s));
  RQ_CUDA(cudaStreamSynchronize(s));
  std::vector<std::complex<double>> lam(nc);
  std::vector<double> et(nc);
  for (int i = 0; i < nc; ++i) {
    const bool first = h1[i] <= h2[i];
    lam[i] = first ? std::complex<double>(r1[2 * i], r1[2 * i + 1])
                   : std::complex<double>(r2[2 * i], r2[2 * i + 1]);
    et[i] = first ? h1[i] : h2[i];
  }
  std::vector<int> order(nc);
  for (int i = 0; i < nc; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    const double dx = std::abs(lam[x] - sh), dy = std::abs(lam[y] - sh);
    if (dx != dy) return dx < dy;
    return lam[x].imag() > lam[y].imag();
  });
  std::vector<double> lsel(2 * (size_t)neig), esel(neig);
  int conv = 0;
  for (int q = 0; q < neig; ++q) {
    const int i = order[q];
    lsel[2 * q] = lam[i].real();
    lsel[2 * q + 1] = lam[i].imag();
    esel[q] = et[i];
    conv += h.est[i] <= E.tol ? 1 : 0;
    RQ_CUDA(cudaMemcpyAsync(X + 2 * N * (int64_t)q, Xa.p + 2 * N * (int64_t)i,
                            sizeof(double) * 2 * N, cudaMemcpyDeviceToDevice, s));
  }
  RQ_CUDA(cudaMemcpyAsync(lambda, lsel.data(), sizeof(double) * 2 * neig, cudaMemcpyHostToDevice, s));
  RQ_CUDA(cudaMemcpyAsync(eta, esel.data(), sizeof(double) * neig, cudaMemcpyHostToDevice, s));
  RQ_CUDA(cudaEventRecord(P.ev1, s));
  DevStatus dst{};
  RQ_CUDA(cudaMemcpyAsync(&dst, P.status.p, sizeof(dst), cudaMemcpyDeviceToHost, s));
  RQ_CUDA(cudaStreamSynchronize(s));
  if (dst.internal)
    throw Error(RIGAQEP_ERR_TIMEOUT, "a bounded wait for a TMA copy of the basis ran out");
  if (dst.timeout)
    throw Error(RIGAQEP_ERR_TIMEOUT, "a bounded wait between the FB work items ran out");
  float ms = 0.f;
  RQ_CUDA(cudaEventElapsedTime(&ms, P.ev0, P.ev1));
  P.info.eigs_ms = ms;
  P.info.n_launches = P.launches;
  P.info.certified = 0;   // no distance certificate for a complex shift
  P.info.cert_margin = -1.0;
  *n_conv = conv;
}

void eigs_run(Problem& P, const EigsParams& E, const double* v1, double* lambda, double* X,
              double* eta, int* n_conv) {
  Plan& L = P.plan;
  cudaStream_t s = P.stream;
  const int m = E.m, nks = E.ncand;
  const double tol = E.tol;
  const int64_t N = L.N, ld = basis_ld(L.N);
  RQ_CUDA(cudaEventRecord(P.ev0, s));
  // in-region calls that differ only in the target (and neig) share the
  // converged candidates of the previous call on the same factor
  if (P.cand_valid && v1 == nullptr && same_candidates(P.cand_E, E)) {
    P.info.n_apply = P.info.n_restarts = P.info.n_spmv = P.info.n_vv = 0;
    P.info.n_qr_sweeps = 0;
    P.info.fb_ms = P.info.ritz_ms = 0.0;
    for (int q = 0; q < 6; ++q) P.info.ritz_phase_cycles[q] = 0.0;
    P.info.reused_candidates = 1;
  } else {
    P.cand_valid = false;
    krylov_schur(P, E, v1);
  }
  if (E.cplx) {
    finish_complex(P, E, lambda, X, eta, n_conv);
    return;
  }
  const RitzOut& h_out = P.cand;
  // the last Ritz step wrote the eigenvectors of H for the candidate values
  // selection of the neig candidates nearest the target (Im > 0 first on
  // ties), and the certificate that no other eigenvalue is nearer
  int neig = E.neig;
  std::vector<int> order(nks);
  for (int i = 0; i < nks; ++i) order[i] = i;
  auto dist = [&](int i) { return std::hypot(h_out.lam[2 * i] - E.target, h_out.lam[2 * i + 1]); };
  auto cls = [&](int i) { double im = h_out.lam[2 * i + 1]; return im > 0 ? 0 : (im == 0 ? 1 : 2); };
  if (E.gep) {
    // undamped pencil: the candidates with mu in [lo, hi), ascending
    std::vector<int> in;
    for (int i = 0; i < nks; ++i)
      if (h_out.lam[2 * i] >= E.lo && h_out.lam[2 * i] < E.hi) in.push_back(i);
    std::stable_sort(in.begin(), in.end(),
                     [&](int a, int b) { return h_out.lam[2 * a] < h_out.lam[2 * b]; });
    P.gep_inside = (int)in.size();
    neig = (int)std::min<size_t>(in.size(), (size_t)E.neig);
    for (int q = 0; q < neig; ++q) order[q] = in[q];
    P.info.certified = 0;
  } else {
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
      double da = dist(a), db = dist(b);
      if (da != db) return da < db;
      return cls(a) < cls(b);
    });
  }
  bool all_conv = true;
  for (int i = 0; i < nks; ++i) all_conv = all_conv && (h_out.est[i] <= tol);
  int sel_conv = 0;
  double dmax = 0.0;
  for (int q = 0; q < neig; ++q) {
    sel_conv += h_out.est[order[q]] <= tol ? 1 : 0;
    dmax = std::max(dmax, dist(order[q]));
  }
  double margin = -1.0;
  bool cert = false;
  if (E.gep) {
    cert = all_conv;   // the count check is the caller's (rigaqep_eigs_undamped)
    margin = 0.0;
  } else if (!E.in_region) {
    cert = all_conv;
    margin = 0.0;
  } else if (all_conv && E.shift >= 0.0 && E.target >= E.shift && P.sigma_min >= 0.0) {
    double r = 0.0;
    for (int i = 0; i < nks; ++i)
      r = std::max(r, std::hypot(h_out.lam[2 * i] - E.shift, h_out.lam[2 * i + 1]));
    double ts = E.target - E.shift;
    double bc = std::sqrt(r * r + ts * (E.target + E.shift + P.sigma_min));
    double br = ts + r;
    double bound = std::min(bc, br);
    margin = bound - dmax;
    cert = bound >= dmax * (1.0 + 1e-12);
  }
  P.info.certified = cert ? 1 : 0;
  P.info.cert_margin = margin;
  if (neig == 0) {   // undamped pencil: no candidate inside the interval
    RQ_CUDA(cudaEventRecord(P.ev1, s));
    RQ_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    RQ_CUDA(cudaEventElapsedTime(&ms, P.ev0, P.ev1));
    P.info.eigs_ms = ms;
    P.info.n_launches = P.launches;
    *n_conv = 0;
    return;
  }
  std::vector<double> lam_sel(2 * neig);
  DBuf<double> Ysel;
  Ysel.alloc(2 * (size_t)m * neig);
  for (int q = 0; q < neig; ++q) {
    int i = order[q];
    lam_sel[2 * q] = h_out.lam[2 * i];
    lam_sel[2 * q + 1] = h_out.lam[2 * i + 1];
    RQ_CUDA(cudaMemcpyAsync(Ysel.p + 2 * (size_t)m * q, P.Y.p + 2 * (size_t)m * i,
                            sizeof(double) * 2 * m, cudaMemcpyDeviceToDevice, s));
  }
  RQ_CUDA(cudaMemcpyAsync(lambda, lam_sel.data(), sizeof(double) * 2 * neig, cudaMemcpyHostToDevice, s));
  {
    size_t smem = sizeof(double) * 2 * (size_t)m * neig;
    smem_at_least((const void*)k_eigvec, smem);
    // the eigenvector is the upper block of the QEP basis, the lower one of
    // the undamped pencil's
    const double* Vb = E.gep ? P.V.p + basis_np(L.N) : P.V.p;
    k_eigvec<<<(unsigned)((N + 127) / 128), 128, smem, s>>>(Vb, ld, m, Ysel.p, neig, P.perm.p, X, N);
    RQ_CUDA(cudaGetLastError());
  }
  DBuf<double> stats;
  stats.alloc(4 * (size_t)neig);
  k_colstats<<<neig, 1024, 0, s>>>(X, N, stats.p);
  RQ_CUDA(cudaGetLastError());
  dim3 g((unsigned)((N + 255) / 256), neig);
  k_colnormalise<<<g, 256, 0, s>>>(X, N, stats.p);
  RQ_CUDA(cudaGetLastError());
  int qb = 2 * P.nsm;
  dim3 gq(qb, neig);
  // residual of the QEP at lambda, or of the undamped pencil: lambda = i sqrt(mu)
  // makes K + lambda^2 M = K - mu M, with the damping term dropped
  const double* lres = lambda;
  DBuf<double> lam_gep;
  if (E.gep) {
    std::vector<double> lg(2 * (size_t)neig, 0.0);
    for (int q = 0; q < neig; ++q) lg[2 * q + 1] = std::sqrt(std::max(0.0, lam_sel[2 * q]));
    lam_gep.upload(lg, s);
    lres = lam_gep.p;
  }
  k_qres<<<gq, 256, 0, s>>>(P.rowptr.p, P.col.p, P.K.p, P.M.p, P.C.p, X, lres, N, P.part.p,
                            E.gep ? 0.0 : 1.0);
  RQ_CUDA(cudaGetLastError());
  k_eta<<<1, 128, 0, s>>>(P.part.p, qb, lres, P.info.norm_K, P.info.norm_M,
                          E.gep ? 0.0 : P.info.norm_C, eta, neig);
  RQ_CUDA(cudaGetLastError());
  P.launches += 5;
  RQ_CUDA(cudaEventRecord(P.ev1, s));
  DevStatus dst{};
  RQ_CUDA(cudaMemcpyAsync(&dst, P.status.p, sizeof(dst), cudaMemcpyDeviceToHost, s));
  RQ_CUDA(cudaStreamSynchronize(s));
  if (dst.internal)
    throw Error(RIGAQEP_ERR_TIMEOUT, "a bounded wait for a TMA copy of the basis ran out");
  if (dst.timeout)
    throw Error(RIGAQEP_ERR_TIMEOUT, "a bounded wait between the FB work items ran out");
  float ms = 0.f;
  RQ_CUDA(cudaEventElapsedTime(&ms, P.ev0, P.ev1));
  P.info.eigs_ms = ms;
  P.info.n_launches = P.launches;
  *n_conv = sel_conv;
}

namespace {
// the element gradients of every pair (templated kernels for p = 2..5)
void launch_grad(Problem& P, int neig, const double* lambda, const double* X, const double* den,
                 double* G) {
  Plan& L = P.plan;
  cudaStream_t s = P.stream;
  const int64_t tot = (int64_t)L.ne * L.ne * neig;
  const unsigned g = (unsigned)((tot + 127) / 128);
  switch (L.p + 1) {
    case 3: k_grad_p<3><<<g, 128, 0, s>>>(X, lambda, den, P.m1.p, P.first_fn.p, L.ne, L.n1, L.N, neig, G); break;
    case 4: k_grad_p<4><<<g, 128, 0, s>>>(X, lambda, den, P.m1.p, P.first_fn.p, L.ne, L.n1, L.N, neig, G); break;
    case 5: k_grad_p<5><<<g, 128, 0, s>>>(X, lambda, den, P.m1.p, P.first_fn.p, L.ne, L.n1, L.N, neig, G); break;
    case 6: k_grad_p<6><<<g, 128, 0, s>>>(X, lambda, den, P.m1.p, P.first_fn.p, L.ne, L.n1, L.N, neig, G); break;
    default:
      k_grad<<<g, 128, 0, s>>>(X, lambda, den, P.m1.p, P.first_fn.p, L.ne, L.p, L.n1, L.N, neig, G);
  }
  RQ_CUDA(cudaGetLastError());
}
}  // namespace

void grad_run(Problem& P, int neig, const double* lambda, const double* X, double* G) {
  Plan& L = P.plan;
  cudaStream_t s = P.stream;
  int64_t N = L.N;
  int nb = 2 * P.nsm;
  DBuf<double> part, den;
  part.alloc(2 * (size_t)nb * neig);
  den.alloc(2 * (size_t)neig);
  dim3 g(nb, neig);
  k_gden<<<g, 256, 0, s>>>(P.rowptr.p, P.col.p, P.M.p, P.C.p, X, lambda, N, part.p);
  RQ_CUDA(cudaGetLastError());
  k_gden_final<<<1, 64, 0, s>>>(part.p, nb, neig, den.p);
  RQ_CUDA(cudaGetLastError());
  launch_grad(P, neig, lambda, X, den.p, G);
  RQ_CUDA(cudaStreamSynchronize(s));
}


// ---- allocation-free variant of the damping sensitivity ----
//
// Scratch for the reduction of x^T (2 lambda M + C) x: per-block partial sums
// (re, im) of up to kNoAllocMaxEig eigenpairs over a fixed grid of
// kNoAllocBlocks blocks (two per SM of a 152-SM GB300; the reduction is
// correct for any SM count), then the denominators.  It
// lives in this file-scope device array, so the call needs no cudaMalloc;
// every GPU that loads the library keeps these 305 KiB until the process
// exits.  Every entry the kernels read is written earlier in the same call.
constexpr int kNoAllocBlocks = 2 * 152;
constexpr int kNoAllocMaxEig = 64;
constexpr size_t kNoAllocScratch = 2 * (size_t)kNoAllocBlocks * kNoAllocMaxEig + 2 * kNoAllocMaxEig;
static __device__ __align__(256) double g_grad_scratch[kNoAllocScratch];

namespace {
std::mutex g_scratch_mu;
double* g_scratch_ptr[256] = {nullptr};

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is queried
// once per device (with that device current) and cached.
double* noalloc_scratch() {
  int dev = 0;
  RQ_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) throw Error(RIGAQEP_ERR_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    RQ_CUDA(cudaGetSymbolAddress(&p, g_grad_scratch));
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  return g_scratch_ptr[dev];
}
}  // namespace

void grad_run_noalloc(Problem& P, int neig, const double* lambda, const double* X, double* G) {
  if (neig < 1 || neig > kNoAllocMaxEig)
    throw Error(RIGAQEP_ERR_ARG, "neig must be in [1, 64] for the allocation-free gradient");
  Plan& L = P.plan;
  cudaStream_t s = P.stream;
  int64_t N = L.N;
  double* part = noalloc_scratch();
  double* den = part + 2 * (size_t)kNoAllocBlocks * kNoAllocMaxEig;
  dim3 g(kNoAllocBlocks, neig);
  k_gden<<<g, 256, 0, s>>>(P.rowptr.p, P.col.p, P.M.p, P.C.p, X, lambda, N, part);
  RQ_CUDA(cudaGetLastError());
  k_gden_final<<<1, 64, 0, s>>>(part, kNoAllocBlocks, neig, den);
  RQ_CUDA(cudaGetLastError());
  int64_t tot = (int64_t)L.ne * L.ne * neig;
  k_grad<<<(unsigned)((tot + 127) / 128), 128, 0, s>>>(X, lambda, den, P.m1.p, P.first_fn.p, L.ne,
                                                       L.p, L.n1, N, neig, G);
  RQ_CUDA(cudaGetLastError());
  RQ_CUDA(cudaStreamSynchronize(s));
}

}  // namespace rq
