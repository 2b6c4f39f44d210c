// Tensor-core front products of the TF32 and BF16 factorisations (tcgen05).
//
// Algorithm 2 ("Factorize Q(s)") factorises every front F = [F11 F21^T;
// F21 F22] of the multifrontal tree.  After the pivot block is factorised
// (F11 = L11 D L11^T) and inverted in place (FP32, SIMT kernels of
// factor.cu), the rest of the front is three dense products:
//   (3) Z   = F21 inv(L11)^T,  L21 = Z D^{-1}      (u x k)
//   (4) U  -= L21 Z^T           (= L21 D L21^T)     (u x u, lower tiles)
//   (5) W   = L21 inv(L11)                          (u x k, FB panel)
// Each is C = A B^T with A (rows x K) and B (cols x K) both K-major, which
// is the operand form of tcgen05.mma.  They run here on the fifth-generation
// tensor cores: 128 x N output tiles (N = 64 or 128), the accumulator in
// tensor memory (TMEM), operands staged in shared memory by TMA
// (cp.async.bulk.tensor) in a three-stage mbarrier pipeline, one elected
// thread issuing the MMAs.
//
// Precision.  A single TF32 (10-bit mantissa) or BF16 (7-bit) product is too
// coarse for FP64 refinement to converge on these fronts, so every operand
// x is split into two terms, x = hi + lo with hi = round(x) and lo =
// round(x - hi), and the product is hi*hi + hi*lo + lo*hi (three MMAs into
// one FP32 accumulator; lo*lo is below the FP32 rounding of the sum for
// TF32).  TF32 terms carry 22 bits, BF16 terms 16 bits.  The BF16 operands
// that scale with the pivots (F21 and Z) are multiplied by a per-front power
// of two 2^-e, e the exponent of the front's largest pivot, so that they sit
// near 1; the epilogue multiplies the products back (exact).
//
// Staged operand layout.  An operand X (n rows x K) is stored in K-blocks of
// RW elements (128 bytes: 32 TF32 / 64 BF16): block b holds rows
// off + b n .. off + b n + n - 1, each row the 128 bytes X[r, b RW ..
// b RW + RW - 1] (zero past K).  One 2-D tensor map over the whole buffer
// (inner dimension RW, one row per 128 bytes) then loads any 128-row (or
// N-row) tile of any front with a box at (0, row) and the 128-byte swizzle,
// which is the canonical K-major SWIZZLE_128B layout that the MMA reads.
// Rows past a front's n inside a box belong to other operands: they only
// reach output rows or columns past the front's extent, which the epilogue
// discards; the K padding inside valid rows is always written as zeros.
#include <cuda_bf16.h>

#include <algorithm>
#include <array>
#include <map>
#include <cstring>
#include <mutex>

#include "internal.h"
#include "tma.cuh"

namespace rq {

namespace {

constexpr int kTcStagesMax = 3;
constexpr uint32_t kTcWaitLimit = 1u << 22;   // polls of a pipeline barrier before giving up
constexpr int kTcThreads = 128;

template <class E>
struct TcElem;
template <>
struct TcElem<float> {
  static constexpr int RW = 32;        // elements per 128-byte row
  static constexpr uint32_t fmt = 2;   // instruction descriptor operand format: TF32
};
template <>
struct TcElem<__nv_bfloat16> {
  static constexpr int RW = 64;
  static constexpr uint32_t fmt = 1;   // BF16 (with .kind::f16)
};

struct TcArgs {
  const TcFront* fr;
  float* Lval;          // FP32 panels
  float* Uval;          // FP32 update blocks
  const float* Dinv;
  const float* Dval;
  float* scale;         // per-front power of two (BF16), else unused
  void* hi;             // staged planes
  void* lo;
  float* C;             // plain product output (mode 0)
  int ldc;
  DevStatus* status;
};

// --- tcgen05 / TMA primitives (inline PTX) ---------------------------------

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// K-major operand tile with the 128-byte swizzle: 8-row groups of 1024 bytes
// (stride byte offset 1024), start address in 16-byte units, descriptor
// version 1 (bits 46-48 = 0b001), swizzle mode 2 (128 bytes) in bits 61-63.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;                 // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
  d |= (uint64_t)1 << 46;                 // descriptor version
  d |= (uint64_t)2 << 61;                 // SWIZZLE_128B
  return d;
}

// Instruction descriptor: FP32 accumulator (bits 4-5 = 1), A and B format
// (bits 7-9, 10-12), both K-major (bits 15, 16 = 0), N / 8 in bits 17-22,
// M / 16 in bits 24-28.
template <class E, int N>
__device__ __forceinline__ uint32_t tc_idesc() {
  return (1u << 4) | (TcElem<E>::fmt << 7) | (TcElem<E>::fmt << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(128 >> 4) << 24);
}

template <class E>
__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t acc);
template <>
__device__ __forceinline__ void tc_mma<float>(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                              uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
template <>
__device__ __forceinline__ void tc_mma<__nv_bfloat16>(uint32_t tmem, uint64_t a, uint64_t b,
                                                      uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// arrives on `bar` when every tcgen05.mma issued so far by this thread completes
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_addr(bar))
               : "memory");
}

// 32 consecutive accumulator columns of this warp's 32 TMEM lanes
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int t = 0; t < 32; ++t) v[t] = __uint_as_float(r[t]);
}

// --- operand splitting -------------------------------------------------------

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t h;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  return __uint_as_float(h);
}
__device__ __forceinline__ void split2(float x, float& hi, float& lo) {
  hi = tf32_round(x);
  lo = tf32_round(x - hi);
}
__device__ __forceinline__ void split2(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// 16 bytes of consecutive elements x[t..] as one vector
__device__ __forceinline__ uint4 pack16(const float* x, int t) {
  return make_uint4(__float_as_uint(x[t]), __float_as_uint(x[t + 1]), __float_as_uint(x[t + 2]),
                    __float_as_uint(x[t + 3]));
}
__device__ __forceinline__ uint32_t bf16_bits(__nv_bfloat16 h) {
  return (uint32_t)__bfloat16_as_ushort(h);
}
__device__ __forceinline__ uint4 pack16(const __nv_bfloat16* x, int t) {
  uint32_t w[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) w[q] = bf16_bits(x[t + 2 * q]) | (bf16_bits(x[t + 2 * q + 1]) << 16);
  return make_uint4(w[0], w[1], w[2], w[3]);
}

// --- kernels -----------------------------------------------------------------

// Per-front power of two for the BF16 operands: 2^-e with e the exponent of
// the largest pivot D_j (one warp per front).
__global__ void k_tc_scale(TcArgs A, const int32_t* fronts, int nf) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= nf) return;
  const int s = fronts[w];
  const TcFront f = A.fr[s];
  float mx = 0.f;
  for (int j = lane; j < f.k; j += 32) mx = fmaxf(mx, fabsf(A.Dval[f.a + j]));
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) A.scale[s] = (mx > 0.f && isfinite(mx)) ? ldexpf(1.f, -ilogbf(mx)) : 1.f;
}

// Staging of the operands of product (3) and (5) from the FP32 panel: one
// CTA per 32-row chunk of one K-block of one operand.  item = {front,
// operand, K-block, first row}; operand 0: F21 (u rows), 1: inv(L11) by rows,
// 2: inv(L11) by columns (row j of the operand = column j of inv(L11)).  The
// pivot block holds inv(L11) strictly below its diagonal; the unit diagonal
// and the zero upper triangle are written explicitly.
template <class E>
__global__ void __launch_bounds__(256) k_tc_stage(TcArgs A, const int4* items, int item_begin,
                                                  int scaled) {
  constexpr int RW = TcElem<E>::RW;
  __shared__ float t[32][RW + 1];
  const int4 it = items[item_begin + blockIdx.x];
  const int s = it.x, which = it.y, b = it.z, r0 = it.w;
  const TcFront f = A.fr[s];
  const int k = f.k, u = f.u;
  const int64_t F = k + u;
  const float* L = A.Lval + f.loff;
  const int nrows = which == 0 ? u : k;
  const int c0 = b * RW;
  const float sc = (which == 0 && scaled) ? A.scale[s] : 1.f;
  for (int q = threadIdx.x; q < 32 * RW; q += blockDim.x) {
    int r, c;
    if (which == 2) {        // contiguous along the operand's columns
      c = q % RW;
      r = q / RW;
    } else {                 // contiguous along the operand's rows
      r = q % 32;
      c = q / 32;
    }
    const int i = r0 + r, j = c0 + c;
    float v = 0.f;
    if (i < nrows && j < k) {
      if (which == 0) v = L[(k + i) + F * j] * sc;
      else if (which == 1) v = j < i ? L[i + F * j] : (j == i ? 1.f : 0.f);
      else v = j > i ? L[j + F * i] : (j == i ? 1.f : 0.f);
    }
    t[r][c] = v;
  }
  __syncthreads();
  E* hi = (E*)A.hi;
  E* lo = (E*)A.lo;
  const int64_t base = which == 0 ? f.offA3 : which == 1 ? f.offB3 : f.offB5;
  for (int q = threadIdx.x; q < 32 * RW; q += blockDim.x) {
    const int c = q % RW, r = q / RW, i = r0 + r;
    if (i < nrows) {
      E h, l;
      split2(t[r][c], h, l);
      const int64_t idx = (base + (int64_t)b * nrows + i) * RW + c;
      hi[idx] = h;
      lo[idx] = l;
    }
  }
}

// Staging of a row-major operand X (nr x K) for the plain product: element
// c of K-block b of row r goes to staged row off + b nr + r (zero past K).
template <class E>
__global__ void k_tc_stage_plain(const float* X, int nr, int K, int64_t off, void* hi_, void* lo_) {
  constexpr int RW = TcElem<E>::RW;
  const int kb = (K + RW - 1) / RW;
  const int64_t n = (int64_t)nr * kb * RW;
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int c = (int)(q % RW);
  const int64_t rb = q / RW;            // staged row within the operand: b nr + r
  const int b = (int)(rb / nr), r = (int)(rb % nr);
  const int j = b * RW + c;
  const float v = j < K ? X[(int64_t)r * K + j] : 0.f;
  E h, l;
  split2(v, h, l);
  ((E*)hi_)[(off + rb) * RW + c] = h;
  ((E*)lo_)[(off + rb) * RW + c] = l;
}

__device__ __forceinline__ void tc_fail(DevStatus* st) { atomicCAS(&st->timeout, 0, 1); }

// One 128 x N output tile C = A B^T per CTA (four warps).  Warp 0 lane 0
// loads K-blocks with TMA into a ring of `stages` buffers, warp 1 lane 0
// issues the MMAs (three per 32-byte K step: hi*hi, hi*lo, lo*hi), and all
// four warps read the accumulator (TMEM lane = tile row) for the epilogue:
//   mode 0: C[i ldc + j] = acc                (plain product)
//   mode 3: Z = scale acc, L21 = Z D^{-1}: both staged as operands of (4), (5)
//   mode 4: U[i + u j] -= scale acc            (tiles on or below the diagonal)
//   mode 5: W[i, j] = acc into the panel       (rows k.., column-major)
// (MODE 45: modes 4 and 5 in one launch, the mode of each tile in its item.)
// Every wait is bounded; on a timeout the CTA records it in the status word,
// waits (bounded) for its own copies and MMAs in flight, frees its TMEM and
// returns without writing.
template <class E, int N, int MODE>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_tc_gemm(TcArgs A, const __grid_constant__ CUtensorMap mAh,
              const __grid_constant__ CUtensorMap mAl, const __grid_constant__ CUtensorMap mBh,
              const __grid_constant__ CUtensorMap mBl, const int4* tiles, int tile_begin,
              int stages) {
  constexpr int RW = TcElem<E>::RW;
  constexpr uint32_t ABYTES = 128 * 128, BBYTES = N * 128;
  constexpr uint32_t STAGE = 2 * ABYTES + 2 * BBYTES;
  extern __shared__ __align__(1024) unsigned char tc_dyn[];
  __shared__ uint64_t full[kTcStagesMax], empty[kTcStagesMax], done;
  __shared__ uint32_t tmem_base;
  __shared__ int err, consumed, issued;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t raw = smem_addr(tc_dyn);
  const uint32_t sbase = (raw + 1023u) & ~1023u;   // 1024-byte aligned ring

  const int4 it = tiles[tile_begin + blockIdx.x];
  const int s = it.x, I0 = it.y, J0 = it.z;
  // mode 45: products (4) and (5) of a level in one launch, the tile's mode in it.w
  const int mode = MODE == 45 ? it.w : MODE;
  const TcFront f = A.fr[s];
  const int u = f.u, k = f.k, kb = f.kb;
  // operands of this mode: A rows nA from offA, B rows nB from offB
  int nA, nB, offA, offB;
  if (mode == 0) { nA = u; nB = f.nB0; offA = f.offA3; offB = f.offB3; }
  else if (mode == 3) { nA = u; nB = k; offA = f.offA3; offB = f.offB3; }
  else if (mode == 4) { nA = u; nB = u; offA = f.offA4; offB = f.offB4; }
  else { nA = u; nB = k; offA = f.offA4; offB = f.offB5; }

  if (tid == 0) {
    for (int q = 0; q < kTcStagesMax; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], 1);
    }
    mbar_init(&done, 1);
    mbar_fence_init();
    err = 0;
    consumed = 0;
    issued = 0;
  }
  __syncwarp();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_base)),
                 "r"((uint32_t)N)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  if (warp == 0 && lane == 0) {
    // producer
    int b = 0;
    for (; b < kb; ++b) {
      const int st = b % stages;
      if (b >= stages && !mbar_wait(&empty[st], (uint32_t)(((b / stages) - 1) & 1), kTcWaitLimit)) {
        err = 1;
        break;
      }
      const uint32_t sa = sbase + st * STAGE;
      uint64_t* fb = &full[st];
      mbar_expect_tx(fb, STAGE);
      const int ra = offA + b * nA + I0, rb = offB + b * nB + J0;
      tma_load_2d_sa(sa, &mAh, 0, ra, fb);
      tma_load_2d_sa(sa + ABYTES, &mAl, 0, ra, fb);
      tma_load_2d_sa(sa + 2 * ABYTES, &mBh, 0, rb, fb);
      tma_load_2d_sa(sa + 2 * ABYTES + BBYTES, &mBl, 0, rb, fb);
    }
    issued = b;
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    const uint32_t idesc = tc_idesc<E, N>();
    int b = 0;
    for (; b < kb; ++b) {
      const int st = b % stages;
      if (!mbar_wait(&full[st], (uint32_t)((b / stages) & 1), kTcWaitLimit)) {
        err = 1;
        break;
      }
      tc_fence_after();
      const uint32_t sa = sbase + st * STAGE;
#pragma unroll
      for (int j = 0; j < 4; ++j) {   // 32-byte K steps of the 128-byte rows
        const uint64_t ah = tc_desc(sa + 32 * j), al = tc_desc(sa + ABYTES + 32 * j);
        const uint64_t bh = tc_desc(sa + 2 * ABYTES + 32 * j);
        const uint64_t bl = tc_desc(sa + 2 * ABYTES + BBYTES + 32 * j);
        tc_mma<E>(tmem, ah, bh, idesc, (b | j) != 0 ? 1u : 0u);
        tc_mma<E>(tmem, ah, bl, idesc, 1u);
        tc_mma<E>(tmem, al, bh, idesc, 1u);
      }
      tc_commit(&empty[st]);   // the stage is free once these MMAs have read it
    }
    consumed = b;
    tc_commit(&done);          // every MMA issued above has completed
  }
  // the accumulator is complete once `done` fires (one thread waits, so
  // that the outcome is uniform across the CTA)
  __shared__ int dflag;
  if (tid == 0) {
    bool ok = mbar_wait(&done, 0, kTcWaitLimit);
    if (!ok) ok = mbar_wait(&done, 0, kTcWaitLimit);   // one more bounded wait before giving up
    dflag = ok ? 1 : 0;
  }
  __syncthreads();
  const bool good = dflag == 1 && err == 0;
  if (!good) {
    if (tid == 0) {
      tc_fail(A.status);
      // copies issued and never consumed still complete on their barriers
      for (int b = consumed; b < issued; ++b)
        mbar_wait(&full[b % stages], (uint32_t)((b / stages) & 1), kTcWaitLimit);
    }
  } else {
    tc_fence_after();
    const int i = I0 + tid;                        // tile row = TMEM lane
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    float sc = 1.f;
    if ((mode == 3 || mode == 4) && A.scale) sc = 1.f / A.scale[s];
    E* hi = (E*)A.hi;
    E* lo = (E*)A.lo;
#pragma unroll 1
    for (int c0 = 0; c0 < N; c0 += 32) {
      const int j0 = J0 + c0;
      if (mode == 3 || mode == 5 || mode == 0) {
        if (j0 >= (mode == 0 ? nB : ((k + RW - 1) / RW) * RW)) break;
      } else if (j0 >= u) {
        break;
      }
      float v[32];
      tc_ld32(lane_base + (uint32_t)c0, v);
      if (mode == 0) {
        if (i < u)
          for (int t = 0; t < 32; ++t)
            if (j0 + t < nB) A.C[(int64_t)i * A.ldc + j0 + t] = v[t];
      } else if (mode == 3) {
        if (i < u) {
          // this chunk is RW-block b = j0 / RW, elements (j0 % RW)..+31; the
          // pivot reciprocals are loaded before any store so that the loads
          // overlap (the stores could alias them as far as the compiler knows)
          const int b = j0 / RW, e0 = j0 % RW;
          float dv[32];
#pragma unroll
          for (int t = 0; t < 32; ++t) dv[t] = j0 + t < k ? __ldg(A.Dinv + f.a + j0 + t) : 0.f;
          const float zs = A.scale ? A.scale[s] : 1.f;
          E lh[32], ll[32], zh[32], zl[32];
#pragma unroll
          for (int t = 0; t < 32; ++t) {
            const float z = j0 + t < k ? v[t] * sc : 0.f;   // unscaled Z (zero past k)
            split2(z * dv[t], lh[t], ll[t]);                // L21 = Z D^{-1}
            split2(z * zs, zh[t], zl[t]);                   // Z staged with the front's scale
          }
          const int64_t ra = ((int64_t)f.offA4 + (int64_t)b * u + i) * RW + e0;
          const int64_t rz = ((int64_t)f.offB4 + (int64_t)b * u + i) * RW + e0;
          // 32 elements per plane and operand, in 16-byte stores
          constexpr int PER = 16 / sizeof(E);
#pragma unroll
          for (int t = 0; t < 32; t += PER) {
            *reinterpret_cast<uint4*>(hi + ra + t) = pack16(lh, t);
            *reinterpret_cast<uint4*>(lo + ra + t) = pack16(ll, t);
            *reinterpret_cast<uint4*>(hi + rz + t) = pack16(zh, t);
            *reinterpret_cast<uint4*>(lo + rz + t) = pack16(zl, t);
          }
        }
      } else if (mode == 4) {
        if (i < u) {
          // all 32 entries are loaded before the first store (see above)
          float* U = A.Uval + f.uoff;
          float old[32];
#pragma unroll
          for (int t = 0; t < 32; ++t) old[t] = j0 + t < u ? U[i + (int64_t)u * (j0 + t)] : 0.f;
#pragma unroll
          for (int t = 0; t < 32; ++t)
            if (j0 + t < u) U[i + (int64_t)u * (j0 + t)] = old[t] - v[t] * sc;
        }
      } else {   // mode 5
        if (i < u) {
          float* P = A.Lval + f.loff;
          const int64_t F = k + u;
          for (int t = 0; t < 32; ++t) {
            const int j = j0 + t;
            if (j < k) P[(k + i) + F * j] = v[t];
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)N)
                 : "memory");
}

template <class E, int N, int MODE>
void launch_gemm(const TcArgs& A, const CUtensorMap* maps, const int32_t* tiles, int begin,
                 int count, int kbmax, cudaStream_t s) {
  if (count <= 0) return;
  constexpr uint32_t STAGE = 2 * 128 * 128 + 2 * N * 128;
  const int stages = std::max(1, std::min(kTcStagesMax, kbmax));
  const size_t smem = (size_t)stages * STAGE + 1024;
  smem_at_least((const void*)k_tc_gemm<E, N, MODE>, smem);
  const CUtensorMap& mB_hi = N == 128 ? maps[0] : maps[2];
  const CUtensorMap& mB_lo = N == 128 ? maps[1] : maps[3];
  k_tc_gemm<E, N, MODE><<<count, kTcThreads, smem, s>>>(A, maps[0], maps[1], mB_hi, mB_lo,
                                                        (const int4*)tiles, begin, stages);
  RQ_CUDA(cudaGetLastError());
}

// Tensor map over a staged plane: rows of 128 bytes (RW elements), boxes of
// RW x box_rows with the 128-byte swizzle; rows past the end read as zeros.
void make_tmap_rows(CUtensorMap* map, void* base, bool bf16, uint64_t rows, uint32_t box_rows) {
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
  const uint32_t rw = bf16 ? 64 : 32;
  cuuint64_t dims[2] = {rw, rows};
  cuuint64_t strides[1] = {128};
  cuuint32_t box[2] = {rw, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                      2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error(RIGAQEP_ERR_CUDA, "cuTensorMapEncodeTiled failed (staged plane)");
}

int kblocks(int K, bool bf16) { return (K + (bf16 ? 64 : 32) - 1) / (bf16 ? 64 : 32); }

// Front-tile autotuner: the width N of the product (3) tiles (64 or 128
// columns) of every level, chosen by timing both on the first factorisation
// of a mesh and precision in the process, then reused.
std::mutex g_tune_mu;
std::map<std::array<int, 6>, std::vector<int32_t>> g_tune;

std::array<int, 6> tune_key(const Plan& L, bool bf16) {
  return {L.ne, L.p, L.block, L.nq, L.leaf_min, bf16 ? 1 : 0};
}

}  // namespace

bool tc_tuning_lookup(const Plan& L, bool bf16, std::vector<int32_t>& n35) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(tune_key(L, bf16));
  if (it == g_tune.end()) return false;
  n35 = it->second;
  return true;
}

void tc_tuning_store(const Plan& L, bool bf16, const std::vector<int32_t>& n35) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[tune_key(L, bf16)] = n35;
}

// Plan of the tensor-core products for precision `bf16` (false: TF32):
// staged-operand offsets of every front (rows counted from the start of its
// level's region; all levels share one buffer), stage items and output tiles
// per level, the two planes and their tensor maps.
void tc_plan(Problem& P, bool bf16) {
  Plan& L = P.plan;
  if (P.tc.ready && P.tc.bf16 == bf16) return;
  std::vector<TcFront> fr(L.nsuper);
  std::vector<int32_t> stage, t3, t3w, t45;
  P.tc.stage_lvl.assign(L.nlevels + 1, 0);
  P.tc.t3_lvl.assign(L.nlevels + 1, 0);
  P.tc.t3w_lvl.assign(L.nlevels + 1, 0);
  P.tc.t45_lvl.assign(L.nlevels + 1, 0);
  P.tc.n35.assign(L.nlevels, 64);
  P.tc.tune_ms.assign(L.nlevels, {0.f, 0.f});
  P.tc.kbmax.assign(L.nlevels, 1);
  int64_t rows_max = 0;
  for (int l = 0; l < L.nlevels; ++l) {
    int64_t row = 0;
    int kmax = 0;
    for (int q = L.lvl_ptr[l]; q < L.lvl_ptr[l + 1]; ++q) kmax = std::max(kmax, L.sptr[L.lvl_nodes[q] + 1] - L.sptr[L.lvl_nodes[q]]);
    P.tc.n35[l] = kmax <= 64 ? 64 : 128;   // until the autotuner has timed both
    P.tc.kbmax[l] = kblocks(kmax, bf16);
    for (int q = L.lvl_ptr[l]; q < L.lvl_ptr[l + 1]; ++q) {
      const int s = L.lvl_nodes[q];
      const int a = L.sptr[s], k = L.sptr[s + 1] - a, u = L.upd_ptr[s + 1] - L.upd_ptr[s];
      const int kb = kblocks(k, bf16);
      TcFront f{};
      f.u = u;
      f.k = k;
      f.kb = kb;
      f.a = a;
      f.loff = L.loff[s];
      f.uoff = L.uoff[s];
      if (u > 0) {
        f.offA3 = (int32_t)row; row += (int64_t)u * kb;
        f.offA4 = (int32_t)row; row += (int64_t)u * kb;
        f.offB4 = (int32_t)row; row += (int64_t)u * kb;
        f.offB3 = (int32_t)row; row += (int64_t)k * kb;
        f.offB5 = (int32_t)row; row += (int64_t)k * kb;
        for (int b = 0; b < kb; ++b) {
          for (int r = 0; r < u; r += 32) stage.insert(stage.end(), {s, 0, b, r});
          for (int r = 0; r < k; r += 32) stage.insert(stage.end(), {s, 1, b, r});
          for (int r = 0; r < k; r += 32) stage.insert(stage.end(), {s, 2, b, r});
        }
        for (int I = 0; I < u; I += 128) {
          for (int J = 0; J < k; J += 64) t3.insert(t3.end(), {s, I, J, 0});
          for (int J = 0; J < k; J += 128) t3w.insert(t3w.end(), {s, I, J, 0});
          for (int J = 0; J <= I; J += 128) t45.insert(t45.end(), {s, I, J, 4});
          for (int J = 0; J < k; J += 128) t45.insert(t45.end(), {s, I, J, 5});
        }
      }
      fr[s] = f;
    }
    if (row >= (int64_t)1 << 31) throw Error(RIGAQEP_ERR_ARG, "front level too large for the staged operands");
    rows_max = std::max(rows_max, row);
    P.tc.stage_lvl[l + 1] = (int32_t)(stage.size() / 4);
    P.tc.t3_lvl[l + 1] = (int32_t)(t3.size() / 4);
    P.tc.t3w_lvl[l + 1] = (int32_t)(t3w.size() / 4);
    P.tc.t45_lvl[l + 1] = (int32_t)(t45.size() / 4);
  }
  cudaStream_t s = P.stream;
  P.tc.fr.alloc(fr.size());
  RQ_CUDA(cudaMemcpyAsync(P.tc.fr.p, fr.data(), fr.size() * sizeof(TcFront), cudaMemcpyHostToDevice, s));
  P.tc.stage.upload(stage, s);
  P.tc.t3.upload(t3, s);
  P.tc.t3w.upload(t3w, s);
  // tile widths chosen earlier for this mesh and precision, if any
  P.tc.tuned = tc_tuning_lookup(L, bf16, P.tc.n35);
  P.tc.t45.upload(t45, s);
  const uint64_t rows = (uint64_t)std::max<int64_t>(rows_max, 128);
  P.tc.hi.alloc(rows * 128);
  P.tc.lo.alloc(rows * 128);
  // padding rows are never written: clear them once so that every value an
  // MMA reads is finite
  RQ_CUDA(cudaMemsetAsync(P.tc.hi.p, 0, rows * 128, s));
  RQ_CUDA(cudaMemsetAsync(P.tc.lo.p, 0, rows * 128, s));
  P.tc.scale.alloc(L.nsuper);
  RQ_CUDA(cudaMemsetAsync(P.tc.scale.p, 0, sizeof(float) * L.nsuper, s));
  make_tmap_rows(&P.tc.maps[0], P.tc.hi.p, bf16, rows, 128);
  make_tmap_rows(&P.tc.maps[1], P.tc.lo.p, bf16, rows, 128);
  make_tmap_rows(&P.tc.maps[2], P.tc.hi.p, bf16, rows, 64);
  make_tmap_rows(&P.tc.maps[3], P.tc.lo.p, bf16, rows, 64);
  P.tc.bf16 = bf16;
  P.tc.ready = true;
}

// Products (3)-(5) of level l on the tensor cores (after its pivot blocks
// are factorised and inverted in FP32).
void launch_tc_level(Problem& P, int l) {
  cudaStream_t s = P.stream;
  const bool bf16 = P.tc.bf16;
  TcArgs A{P.tc.fr.p, P.Lval32.p, P.Uval32.p, P.Dinv32.p, P.Dval32.p,
           bf16 ? P.tc.scale.p : nullptr, P.tc.hi.p, P.tc.lo.p, nullptr, 0, P.status.p};
  const int sb = P.tc.stage_lvl[l], sc = P.tc.stage_lvl[l + 1] - sb;
  if (sc == 0) return;
  const Plan& L = P.plan;
  if (bf16) {
    const int nf = L.lvl_ptr[l + 1] - L.lvl_ptr[l];
    k_tc_scale<<<(nf + 7) / 8, 256, 0, s>>>(A, P.lvl_nodes.p + L.lvl_ptr[l], nf);
    RQ_CUDA(cudaGetLastError());
    ++P.launches;
  }
  if (bf16) k_tc_stage<__nv_bfloat16><<<sc, 256, 0, s>>>(A, (const int4*)P.tc.stage.p, sb, 1);
  else k_tc_stage<float><<<sc, 256, 0, s>>>(A, (const int4*)P.tc.stage.p, sb, 0);
  RQ_CUDA(cudaGetLastError());
  ++P.launches;
  const int kbm = P.tc.kbmax[l];
  const int b3 = P.tc.t3_lvl[l], c3 = P.tc.t3_lvl[l + 1] - b3;
  const int b3w = P.tc.t3w_lvl[l], c3w = P.tc.t3w_lvl[l + 1] - b3w;
  const int b45 = P.tc.t45_lvl[l], c45 = P.tc.t45_lvl[l + 1] - b45;
  const CUtensorMap* mp = P.tc.maps;
  auto product3 = [&](int n) {
    if (bf16) {
      if (n == 64) launch_gemm<__nv_bfloat16, 64, 3>(A, mp, P.tc.t3.p, b3, c3, kbm, s);
      else launch_gemm<__nv_bfloat16, 128, 3>(A, mp, P.tc.t3w.p, b3w, c3w, kbm, s);
    } else {
      if (n == 64) launch_gemm<float, 64, 3>(A, mp, P.tc.t3.p, b3, c3, kbm, s);
      else launch_gemm<float, 128, 3>(A, mp, P.tc.t3w.p, b3w, c3w, kbm, s);
    }
  };
  if (!P.tc.tuned) {
    // autotuner: time both tile widths (the product is idempotent: the second
    // run rewrites the same staged L21 and Z), keep the faster
    cudaEvent_t e[3];
    for (auto& ev : e) RQ_CUDA(cudaEventCreate(&ev));
    RQ_CUDA(cudaEventRecord(e[0], s));
    product3(64);
    RQ_CUDA(cudaEventRecord(e[1], s));
    product3(128);
    RQ_CUDA(cudaEventRecord(e[2], s));
    RQ_CUDA(cudaEventSynchronize(e[2]));
    float t64 = 0.f, t128 = 0.f;
    RQ_CUDA(cudaEventElapsedTime(&t64, e[0], e[1]));
    RQ_CUDA(cudaEventElapsedTime(&t128, e[1], e[2]));
    for (auto& ev : e) RQ_CUDA(cudaEventDestroy(ev));
    P.tc.n35[l] = t128 < t64 ? 128 : 64;
    P.tc.tune_ms[l] = {t64, t128};
    P.launches += 2;
  } else {
    product3(P.tc.n35[l]);
    ++P.launches;
  }
  if (bf16) launch_gemm<__nv_bfloat16, 128, 45>(A, mp, P.tc.t45.p, b45, c45, kbm, s);
  else launch_gemm<float, 128, 45>(A, mp, P.tc.t45.p, b45, c45, kbm, s);
  ++P.launches;
}

// After the first tensor-core factorisation of a mesh: keep its tile widths.
void tc_tuning_done(Problem& P) {
  if (P.tc.tuned) return;
  P.tc.tuned = true;
  tc_tuning_store(P.plan, P.tc.bf16, P.tc.n35);
}

// Plain product C = A B^T (A m x K, B n x K, C m x n, all row-major FP32 on
// the device) through the same staging and tensor-core kernels: the operands
// are split into two terms and staged into K-blocks, one tile per 128 x 128
// block of C.  Used to check the products in isolation.
void tc_plain_gemm(int m, int n, int K, const float* Ad, const float* Bd, float* Cd, bool bf16,
                   cudaStream_t s) {
  const int RW = bf16 ? 64 : 32;
  const int kb = kblocks(K, bf16);
  const int64_t rowsA = (int64_t)m * kb, rowsB = (int64_t)n * kb;
  const int64_t rows = std::max<int64_t>(rowsA + rowsB, 128);
  if (rows >= (int64_t)1 << 31) throw Error(RIGAQEP_ERR_ARG, "product too large");
  DBuf<unsigned char> hi, lo;
  hi.alloc(rows * 128);
  lo.alloc(rows * 128);
  RQ_CUDA(cudaMemsetAsync(hi.p, 0, rows * 128, s));
  RQ_CUDA(cudaMemsetAsync(lo.p, 0, rows * 128, s));
  const unsigned ga = (unsigned)std::max<int64_t>(1, (rowsA * RW + 255) / 256);
  const unsigned gb = (unsigned)std::max<int64_t>(1, (rowsB * RW + 255) / 256);
  if (bf16) {
    k_tc_stage_plain<__nv_bfloat16><<<ga, 256, 0, s>>>(Ad, m, K, 0, hi.p, lo.p);
    k_tc_stage_plain<__nv_bfloat16><<<gb, 256, 0, s>>>(Bd, n, K, rowsA, hi.p, lo.p);
  } else {
    k_tc_stage_plain<float><<<ga, 256, 0, s>>>(Ad, m, K, 0, hi.p, lo.p);
    k_tc_stage_plain<float><<<gb, 256, 0, s>>>(Bd, n, K, rowsA, hi.p, lo.p);
  }
  RQ_CUDA(cudaGetLastError());
  TcFront f{};
  f.u = m;
  f.k = K;
  f.kb = kb;
  f.nB0 = n;
  f.offA3 = 0;
  f.offB3 = (int32_t)rowsA;
  DBuf<TcFront> fr;
  fr.alloc(1);
  RQ_CUDA(cudaMemcpyAsync(fr.p, &f, sizeof(f), cudaMemcpyHostToDevice, s));
  std::vector<int32_t> tiles;
  for (int I = 0; I < m; I += 128)
    for (int J = 0; J < n; J += 128) tiles.insert(tiles.end(), {0, I, J, 0});
  DBuf<int32_t> td;
  td.upload(tiles, s);
  DBuf<DevStatus> st;
  st.alloc(1);
  RQ_CUDA(cudaMemsetAsync(st.p, 0, sizeof(DevStatus), s));
  CUtensorMap maps[4];
  make_tmap_rows(&maps[0], hi.p, bf16, rows, 128);
  make_tmap_rows(&maps[1], lo.p, bf16, rows, 128);
  make_tmap_rows(&maps[2], hi.p, bf16, rows, 64);
  make_tmap_rows(&maps[3], lo.p, bf16, rows, 64);
  TcArgs A{fr.p, nullptr, nullptr, nullptr, nullptr, nullptr, hi.p, lo.p, Cd, n, st.p};
  const int nt = (int)(tiles.size() / 4);
  if (bf16) launch_gemm<__nv_bfloat16, 128, 0>(A, maps, td.p, 0, nt, kb, s);
  else launch_gemm<float, 128, 0>(A, maps, td.p, 0, nt, kb, s);
  DevStatus h;
  RQ_CUDA(cudaMemcpyAsync(&h, st.p, sizeof(h), cudaMemcpyDeviceToHost, s));
  RQ_CUDA(cudaStreamSynchronize(s));
  if (h.timeout) throw Error(RIGAQEP_ERR_TIMEOUT, "a bounded wait of the tensor-core pipeline ran out");
}

}  // namespace rq
