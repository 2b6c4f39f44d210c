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
// Factorisation, per tree level (all fronts of a level together): (1) one CTA
// per front zeroes the front, places the original entries of the pivot
// columns and extend-adds the children's U blocks; (2) one CTA per front
// factorises the k x k pivot block (LDL^T) and inverts L11; then, spread over
// many CTAs, (3) L21 = F21 inv(L11)^T D^{-1} in 16-row chunks, (4) the Schur
// complement U -= L21 D L21^T in 32 x 32 tiles and (5) W = L21 inv(L11).
//
// Partitioned inverse: at the end of each front's factorisation the unit-lower
// pivot block L11 is replaced by inv(L11) and L21 by W = L21 inv(L11), so a
// front's forward elimination is one matrix-vector product with the panel
// [inv(L11); W] and its backward elimination one transposed product with the
// same panel; no front has a sequential substitution chain.
//
// FB, one launch per level and sweep.  Forward (leaves first): work items of
// 32 panel rows; each gathers its front's right-hand side and children's
// update vectors, then forms D^{-1} inv(L11) x_s (pivot rows) or the update
// vector y_s = children - W x_s (update rows).  Backward (root first): work
// items of 32 pivot columns form x_s = inv(L11)^T D^{-1}z - W^T x_struct.
#include "internal.h"

#include <cooperative_groups.h>
#include <type_traits>

#include "cplx.cuh"

#include <cmath>

namespace rq {
namespace {

template <class T>
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
  T* Lval;
  T* Uval;
  T* Dinv;
  T* Dval;
  DevStatus* status;
  int indef;   // 1: pivots of either sign (count the negative ones), 0: SPD
};

// complex storage (double2 pairs) as the kernels' scalar type
inline zd* zp(double2* p) { return reinterpret_cast<zd*>(p); }

template <class T>
FrontArgs<T> front_args(Problem& P);
template <>
FrontArgs<double> front_args<double>(Problem& P) {
  return FrontArgs<double>{P.sptr.p,      P.upd_ptr.p, P.upd_idx.p, P.relmap.p, P.child_ptr.p,
                           P.child_idx.p, P.lvl_nodes.p, P.loff.p,  P.uoff.p,   P.Lval.p,
                           P.Uval.p,      P.Dinv.p,    P.Dval.p,    P.status.p, 0};
}
template <>
FrontArgs<zd> front_args<zd>(Problem& P) {
  return FrontArgs<zd>{P.sptr.p,      P.upd_ptr.p,   P.upd_idx.p, P.relmap.p, P.child_ptr.p,
                       P.child_idx.p, P.lvl_nodes.p, P.loff.p,    P.uoff.p,   zp(P.cx.Lval.p),
                       zp(P.cx.Uval.p), zp(P.cx.Dinv.p), zp(P.cx.Dval.p), P.status.p, 0};
}
template <>
FrontArgs<float> front_args<float>(Problem& P) {
  return FrontArgs<float>{P.sptr.p,      P.upd_ptr.p, P.upd_idx.p, P.relmap.p, P.child_ptr.p,
                          P.child_idx.p, P.lvl_nodes.p, P.loff.p,  P.uoff.p,   P.Lval32.p,
                          P.Uval32.p,    P.Dinv32.p,  P.Dval32.p,  P.status.p, 0};
}

// Assembly of the fronts of one level: nsplit CTAs per front, CTA `part`
// owning the front columns [part F / nsplit, (part + 1) F / nsplit).  Every
// front entry belongs to one column, so the CTAs of a front never write the
// same entry; each zeroes its columns of the panel L (pivot columns) and of
// the update block U, scatters the original entries of its pivot columns,
// and adds the children's update blocks in child order (the child columns
// that map into its range are contiguous: relmap is increasing).
template <class T>
__global__ void k_front_assemble(FrontArgs<T> A, int lvl_begin, int nsplit,
                                 const int32_t* rowptr_n, const int32_t* fpos, const double* Kn,
                                 const double* Mn, const double* Cn, double s2, double s1,
                                 double s2i, double s1i) {
  const int f = blockIdx.x / nsplit, part = blockIdx.x % nsplit;
  int s = A.lvl_nodes[lvl_begin + f];
  int a = A.sptr[s], k = A.sptr[s + 1] - a;
  int u = A.upd_ptr[s + 1] - A.upd_ptr[s];
  int64_t F = k + u;
  const int c_lo = (int)(F * part / nsplit), c_hi = (int)(F * (part + 1) / nsplit);
  T* L = A.Lval + A.loff[s];
  T* U = A.Uval + A.uoff[s];
  // zero the owned columns
  const int lk_lo = min(c_lo, k), lk_hi = min(c_hi, k);          // pivot columns
  const int uk_lo = max(c_lo, k) - k, uk_hi = max(c_hi, k) - k;  // update-block columns
  for (int64_t i = threadIdx.x; i < F * (lk_hi - lk_lo); i += blockDim.x) L[F * lk_lo + i] = T(0);
  for (int64_t i = threadIdx.x; i < (int64_t)u * (uk_hi - uk_lo); i += blockDim.x)
    U[(int64_t)u * uk_lo + i] = T(0);
  __syncthreads();
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int t = lk_lo + warp; t < lk_hi; t += nw) {
    int j = a + t;
    for (int32_t q = rowptr_n[j] + lane; q < rowptr_n[j + 1]; q += 32) {
      int pos = fpos[q];
      if (pos >= 0)
        L[pos + F * t] = from_parts<T>(s2 * Mn[q] + s1 * Cn[q] + Kn[q], s2i * Mn[q] + s1i * Cn[q]);
    }
  }
  __syncthreads();
  for (int ci = A.child_ptr[s]; ci < A.child_ptr[s + 1]; ++ci) {
    int c = A.child_idx[ci];
    int uc = A.upd_ptr[c + 1] - A.upd_ptr[c];
    const int32_t* rm = A.relmap + A.upd_ptr[c];
    const T* Uc = A.Uval + A.uoff[c];
    // child columns q with rm[q] in [c_lo, c_hi)
    int q_lo = 0, h = uc;
    while (q_lo < h) {
      const int mid = (q_lo + h) >> 1;
      if (rm[mid] < c_lo) q_lo = mid + 1;
      else h = mid;
    }
    int q_hi = q_lo;
    h = uc;
    while (q_hi < h) {
      const int mid = (q_hi + h) >> 1;
      if (rm[mid] < c_hi) q_hi = mid + 1;
      else h = mid;
    }
    for (int q = q_lo + warp; q < q_hi; q += nw) {
      int pc = rm[q];
      for (int r = q + lane; r < uc; r += 32) {
        int pr = rm[r];
        T v = Uc[r + (int64_t)uc * q];
        if (pc < k) L[pr + F * pc] += v;
        else U[(pr - k) + (int64_t)u * (pc - k)] += v;
      }
    }
    __syncthreads();
  }
}

// Pivot block of one front (one CTA): right-looking LDL^T of the k x k
// pivot block (rows < k only), D and D^{-1} stored, then inv(L11) in place
// (unit lower; column j from the already inverted trailing block, last
// column first, staged in shared memory).
template <class T>
__global__ void k_pivot_factor(FrontArgs<T> A, const int32_t* fronts) {
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  T* lb = reinterpret_cast<T*>(dyn_smem);
  __shared__ T dsh, rdsh;   // pivot and its reciprocal (one FP64 division per pivot)
  int s = fronts[blockIdx.x];
  int a = A.sptr[s], k = A.sptr[s + 1] - a;
  int u = A.upd_ptr[s + 1] - A.upd_ptr[s];
  int64_t F = k + u;
  T* L = A.Lval + A.loff[s];
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int t = 0; t < k; ++t) {
    if (threadIdx.x == 0) {
      T d = L[t + F * t];
      if (pivot_bad(d, A.indef)) {
        atomicCAS(&A.status->pivot_fail, 0, s + 1);
        d = T(1);  // keep going with a harmless value; the host reports the failure
      } else if (pivot_negative(d)) {
        atomicAdd(&A.status->neg_pivots, 1);
      }
      dsh = d;
      rdsh = T(1) / d;
      L[t + F * t] = T(1);
      A.Dinv[a + t] = rdsh;
      A.Dval[a + t] = d;
    }
    __syncthreads();
    T d = dsh;
    T rd = rdsh;
    for (int i = t + 1 + threadIdx.x; i < k; i += blockDim.x) {
      T l = L[i + F * t] * rd;
      lb[i] = l;
      L[i + F * t] = l;
    }
    __syncthreads();
    for (int c = t + 1 + warp; c < k; c += nw) {
      T lc = d * lb[c];
      for (int i = c + lane; i < k; i += 32) L[i + F * c] -= lb[i] * lc;
    }
    __syncthreads();
  }
  for (int j = k - 2; j >= 0; --j) {
    for (int i = j + 1 + threadIdx.x; i < k; i += blockDim.x) {
      T v0 = 0.0, v1 = T(0);
      int c = j + 1;
      for (; c + 1 < i; c += 2) {
        v0 -= L[i + F * c] * L[c + F * j];
        v1 -= L[i + F * (c + 1)] * L[(c + 1) + F * j];
      }
      for (; c < i; ++c) v0 -= L[i + F * c] * L[c + F * j];
      lb[i] = (v0 + v1) - L[i + F * j];      // the c = i term, inv(L11)[i, i] = 1
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < k; i += blockDim.x) L[i + F * j] = lb[i];
    __syncthreads();
  }
}

// Pivot block of one large front by a cluster of CTAs (one front per
// cluster; the block lives in global memory, L2-resident, and the cluster
// barriers order it between the CTAs; values written by another CTA are read
// through L2):
//  LDL^T by 32-column panels: CTA 0 factors the panel (all rows below it) in
//  shared memory and writes it back with D; then every CTA takes 32 x 32
//  tiles of the trailing lower triangle, A -= L_panel D L_panel^T.
//  inv(L11) by 32-column blocks from the last:
//    X[rest, J] = -X[rest, rest] L[rest, J] X_JJ,   X_JJ = inv(L_JJ),
//  with X[rest, rest] already in place; every CTA inverts the 32 x 32 block
//  itself (forward elimination on the identity), reads L[rest, J] before any
//  CTA overwrites it, and forms every CTA-th row of the result.
constexpr int kClusterCTAs = 8;
constexpr int kClusterMinK = 64;    // pivot blocks from this size use a cluster
constexpr int kClusterMaxK = 800;   // up to this size (k x 32 panel in shared memory)
constexpr int kClusterMaxKc = 384;  // the same for the complex factor (16-byte scalars)
constexpr size_t kSmemOptIn = 227 * 1024;   // largest dynamic shared memory of a CTA
// largest row panel of k_panel_rows in shared memory (its static tiles take
// the rest of the opt-in size)
constexpr size_t kPanelSmemMax = 200 * 1024;

template <class T>
__global__ void __launch_bounds__(256) k_pivot_cluster(FrontArgs<T> A, const int32_t* fronts) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int CS = (int)cl.num_blocks();
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  T* Y = reinterpret_cast<T*>(dyn_smem);   // rows x 32, column-major (ld = rows)
  __shared__ T bl[32][33];                 // L_JJ
  __shared__ T bx[32][33];                 // inv(L_JJ)
  __shared__ T dv[32];
  __shared__ T rdv;                        // 1 / pivot, formed once
  const int s = fronts[blockIdx.x / CS];
  const int a = A.sptr[s], k = A.sptr[s + 1] - a;
  const int u = A.upd_ptr[s + 1] - A.upd_ptr[s];
  const int64_t F = k + u;
  T* L = A.Lval + A.loff[s];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // ---- LDL^T by panels
  for (int j0 = 0; j0 < k; j0 += 32) {
    const int jb = min(32, k - j0);
    const int R = k - j0;
    if (rank == 0) {
      for (int q = tid; q < R * jb; q += 256) {
        int r = q % R, c = q / R;
        Y[r + R * c] = __ldcg(L + (j0 + r) + F * (j0 + c));
      }
      __syncthreads();
      for (int t = 0; t < jb; ++t) {
        if (tid == 0) {
          T d = Y[t + R * t];
          if (pivot_bad(d, A.indef)) {
            atomicCAS(&A.status->pivot_fail, 0, s + 1);
            d = T(1);  // keep going with a harmless value; the host reports the failure
          } else if (pivot_negative(d)) {
            atomicAdd(&A.status->neg_pivots, 1);
          }
          dv[t] = d;
          rdv = T(1) / d;
        }
        __syncthreads();
        const T d = dv[t], rd = rdv;
        for (int r = t + 1 + tid; r < R; r += 256) Y[r + R * t] *= rd;
        __syncthreads();
        for (int c = t + 1 + warp; c < jb; c += 8) {
          const T f = d * Y[c + R * t];
          for (int r = c + lane; r < R; r += 32) Y[r + R * c] -= Y[r + R * t] * f;
        }
        __syncthreads();
      }
      for (int q = tid; q < R * jb; q += 256) {
        int r = q % R, c = q / R;
        if (r >= c) L[(j0 + r) + F * (j0 + c)] = r == c ? T(1) : Y[r + R * c];
      }
      for (int t = tid; t < jb; t += 256) {
        A.Dval[a + j0 + t] = dv[t];
        A.Dinv[a + j0 + t] = T(1) / dv[t];
      }
    }
    cl.sync();
    const int Rt = k - j0 - jb;    // trailing rows and columns
    if (Rt > 0) {
      for (int q = tid; q < Rt * jb; q += 256) {
        int r = q % Rt, c = q / Rt;
        Y[r + Rt * c] = __ldcg(L + (j0 + jb + r) + F * (j0 + c));
      }
      if (tid < jb) dv[tid] = __ldcg(A.Dval + a + j0 + tid);
      __syncthreads();
      const int nt = (Rt + 31) / 32;
      int tile = 0;
      for (int I = 0; I < nt; ++I)
        for (int J = 0; J <= I; ++J, ++tile) {
          if (tile % CS != rank) continue;
          const int c = J * 32 + lane;
          for (int p = 0; p < 4; ++p) {
            const int r = I * 32 + warp + 8 * p;
            if (r < Rt && c < Rt && r >= c) {
              T acc = T(0);
              for (int t = 0; t < jb; ++t) acc += Y[r + Rt * t] * (dv[t] * Y[c + Rt * t]);
              T* dst = L + (j0 + jb + r) + F * (j0 + jb + c);
              *dst = __ldcg(dst) - acc;
            }
          }
        }
    }
    cl.sync();
  }
  // ---- inv(L11) in place, blocks from the last
  const int nb = (k + 31) / 32;
  for (int J = nb - 1; J >= 0; --J) {
    const int j0 = J * 32, jb = min(32, k - j0);
    const int Rr = k - j0 - jb;
    for (int q = tid; q < 32 * 32; q += 256) {
      int r = q & 31, c = q >> 5;
      bl[r][c] = (r < jb && c < r) ? __ldcg(L + (j0 + r) + F * (j0 + c)) : T(0);
      bx[r][c] = r == c ? T(1) : T(0);
    }
    for (int q = tid; q < Rr * jb; q += 256) {
      int r = q % Rr, c = q / Rr;
      Y[r + Rr * c] = __ldcg(L + (j0 + jb + r) + F * (j0 + c));
    }
    __syncthreads();
    // forward elimination on the identity: after step t, row t of bx is final
    for (int t = 0; t < jb; ++t) {
      for (int q = tid; q < 32 * 32; q += 256) {
        int r = q & 31, c = q >> 5;
        if (r > t && r < jb && c <= t) bx[r][c] -= bl[r][t] * bx[t][c];
      }
      __syncthreads();
    }
    cl.sync();   // every CTA holds L[rest, J] before any overwrites it
    for (int i = rank + CS * warp; i < Rr; i += CS * 8) {
      // z = Y[i, :] + sum_{q < i} X[i, q] Y[q, :]   (lane = column)
      T z = lane < jb ? Y[i + Rr * lane] : T(0);
      const T* xi = L + (j0 + jb + i) + F * (int64_t)(j0 + jb);
      const int lc = lane < jb ? lane : 0;
      const T lm = lane < jb ? T(1) : T(0);
      int q = 0;
      for (; q + 8 <= i; q += 8) {   // eight row entries of X in flight
        T xv[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) xv[t] = __ldcg(xi + F * (q + t));
#pragma unroll
        for (int t = 0; t < 8; ++t) z += xv[t] * (lm * Y[(q + t) + Rr * lc]);
      }
      for (; q < i; ++q) z += __ldcg(xi + F * q) * (lm * Y[q + Rr * lc]);
      // X[i, J] = -z X_JJ:  out[c] = -sum_{t >= c} z[t] bx[t][c]
      T o = T(0);
      for (int t = 0; t < jb; ++t) {
        T zt = __shfl_sync(0xffffffffu, z, t);
        if (t >= lane) o += zt * bx[t][lane];
      }
      if (lane < jb) L[(j0 + jb + i) + F * (j0 + lane)] = -o;
    }
    if (rank == 0)
      for (int q = tid; q < jb * jb; q += 256) {
        int r = q % jb, c = q / jb;
        if (r > c) L[(j0 + r) + F * (j0 + c)] = bx[r][c];
      }
    cl.sync();
  }
}

// Pivot blocks wider than the cluster kernel holds (k x 32 panel beyond
// shared memory), by 32-column blocks over many CTAs, one launch per step:
//   LDL^T, for each block column J from the first:
//     diag:   A_JJ = L_JJ D_J L_JJ^T (one CTA per front), X_JJ = inv(L_JJ)
//             kept for the next step;
//     panel:  L_IJ = A_IJ X_JJ^T D_J^{-1} for every 32-row block I below;
//     update: A_IK -= L_IJ D_J L_KJ^T for the lower tiles I >= K below J;
//   inv(L11), for each J from the last:
//     inv:    X[I, J] = -(L_IJ + sum_{J < Q <= I} X_IQ L_QJ) X_JJ for the
//             blocks I below J (X below J is final), into a buffer;
//     store:  the buffer into column block J, X_JJ onto its diagonal block.
// Each launch covers every wide front of the level (blockIdx.x = front); the
// fronts' pivot blocks live in global memory (the panel storage), and the
// kernel boundaries order the steps.  Entries above the diagonal are never
// written (the FB's triangle relies on their being zero).
constexpr int kWideB = 32;
constexpr int kWideFromK = 256;   // pivot blocks above this size take the wide path (measured: faster than the cluster)

template <class T>
struct WideFront {
  T* L;      // pivot block, column-major, leading dimension F
  int64_t F;
  int a, k;  // first pivot (global index) and pivot count
};
template <class T>
__device__ __forceinline__ WideFront<T> wide_front(const FrontArgs<T>& A, const int32_t* fl, int f) {
  const int s = fl[f];
  WideFront<T> w;
  w.a = A.sptr[s];
  w.k = A.sptr[s + 1] - w.a;
  w.F = w.k + (A.upd_ptr[s + 1] - A.upd_ptr[s]);
  w.L = A.Lval + A.loff[s];
  return w;
}

// inv of the unit lower 32 x 32 block bl (rows/cols < jb) into bx, by forward
// elimination on the identity (all threads of the CTA)
template <class T>
__device__ void unit_lower_inverse(const T (*bl)[33], T (*bx)[33], int jb) {
  for (int q = threadIdx.x; q < 32 * 32; q += blockDim.x) {
    const int r = q & 31, c = q >> 5;
    bx[r][c] = r == c ? T(1) : T(0);
  }
  __syncthreads();
  for (int t = 0; t < jb; ++t) {
    for (int q = threadIdx.x; q < 32 * 32; q += blockDim.x) {
      const int r = q & 31, c = q >> 5;
      if (r > t && r < jb && c <= t) bx[r][c] -= bl[r][t] * bx[t][c];
    }
    __syncthreads();
  }
}

template <class T>
__global__ void __launch_bounds__(256) k_wide_diag(FrontArgs<T> A, const int32_t* fl, int j0,
                                                   T* xjj) {
  const WideFront<T> w = wide_front(A, fl, blockIdx.x);
  if (j0 >= w.k) return;
  const int jb = min(kWideB, w.k - j0);
  __shared__ T bl[32][33], bx[32][33];
  __shared__ T dsh, rdsh;
  for (int q = threadIdx.x; q < 32 * 32; q += blockDim.x) {
    const int r = q & 31, c = q >> 5;
    bl[r][c] = (r < jb && c < jb && r >= c) ? w.L[(j0 + r) + w.F * (j0 + c)] : T(0);
  }
  __syncthreads();
  for (int t = 0; t < jb; ++t) {
    if (threadIdx.x == 0) {
      T d = bl[t][t];
      if (pivot_bad(d, A.indef)) {
        atomicCAS(&A.status->pivot_fail, 0, fl[blockIdx.x] + 1);
        d = T(1);  // keep going with a harmless value; the host reports the failure
      } else if (pivot_negative(d)) {
        atomicAdd(&A.status->neg_pivots, 1);
      }
      dsh = d;
      rdsh = T(1) / d;
      A.Dval[w.a + j0 + t] = d;
      A.Dinv[w.a + j0 + t] = rdsh;
    }
    __syncthreads();
    const T d = dsh, rd = rdsh;
    if (threadIdx.x > t && threadIdx.x < jb) bl[threadIdx.x][t] *= rd;
    __syncthreads();
    for (int q = threadIdx.x; q < 32 * 32; q += blockDim.x) {
      const int r = q & 31, c = q >> 5;
      if (c > t && r >= c && r < jb) bl[r][c] -= bl[r][t] * (d * bl[c][t]);
    }
    __syncthreads();
  }
  for (int q = threadIdx.x; q < 32 * 32; q += blockDim.x) {
    const int r = q & 31, c = q >> 5;
    if (r < jb && c < jb && r >= c) w.L[(j0 + r) + w.F * (j0 + c)] = r == c ? T(1) : bl[r][c];
  }
  unit_lower_inverse(bl, bx, jb);
  T* X = xjj + (size_t)blockIdx.x * 32 * 32;
  for (int q = threadIdx.x; q < 32 * 32; q += blockDim.x) X[q] = bx[q & 31][q >> 5];
}

// L_IJ = A_IJ X_JJ^T D_J^{-1} for the 32-row block I = blockIdx.y below J
template <class T>
__global__ void __launch_bounds__(256) k_wide_panel(FrontArgs<T> A, const int32_t* fl, int j0,
                                                    const T* xjj) {
  const WideFront<T> w = wide_front(A, fl, blockIdx.x);
  if (j0 >= w.k) return;
  const int jb = min(kWideB, w.k - j0);
  const int i0 = j0 + jb + kWideB * (int)blockIdx.y;
  if (i0 >= w.k) return;
  const int ib = min(kWideB, w.k - i0);
  __shared__ T ya[32][33], bx[32][33];
  __shared__ T dinv[32];
  const T* X = xjj + (size_t)blockIdx.x * 32 * 32;
  for (int q = threadIdx.x; q < 32 * 32; q += blockDim.x) {
    const int r = q & 31, c = q >> 5;
    ya[r][c] = (r < ib && c < jb) ? w.L[(i0 + r) + w.F * (j0 + c)] : T(0);
    bx[r][c] = X[q];
  }
  if (threadIdx.x < jb) dinv[threadIdx.x] = A.Dinv[w.a + j0 + threadIdx.x];
  __syncthreads();
  for (int q = threadIdx.x; q < 32 * 32; q += blockDim.x) {
    const int r = q & 31, c = q >> 5;   // out[r][c] = dinv[c] sum_{t <= c} A[r][t] X[c][t]
    if (r < ib && c < jb) {
      T acc = T(0);
      for (int t = 0; t <= c; ++t) acc += ya[r][t] * bx[c][t];
      w.L[(i0 + r) + w.F * (j0 + c)] = acc * dinv[c];
    }
  }
}

// A_IK -= L_IJ D_J L_KJ^T for the lower tile (I, K) = tile blockIdx.y of the
// trailing block below J (tiles numbered row by row: I(I+1)/2 + K)
template <class T>
__global__ void __launch_bounds__(256) k_wide_update(FrontArgs<T> A, const int32_t* fl, int j0) {
  const WideFront<T> w = wide_front(A, fl, blockIdx.x);
  if (j0 >= w.k) return;
  const int jb = min(kWideB, w.k - j0);
  const int t0 = j0 + jb, R = w.k - t0;
  const int nt = (R + kWideB - 1) / kWideB;
  const int tile = (int)blockIdx.y;
  if (tile >= nt * (nt + 1) / 2) return;
  int I = (int)((sqrt(8.0 * tile + 1.0) - 1.0) * 0.5);
  while (I * (I + 1) / 2 > tile) --I;
  while ((I + 1) * (I + 2) / 2 <= tile) ++I;
  const int K = tile - I * (I + 1) / 2;
  const int ri = t0 + kWideB * I, ck = t0 + kWideB * K;
  __shared__ T li[32][33], lk[32][33];
  __shared__ T dv[32];
  for (int q = threadIdx.x; q < 32 * 32; q += blockDim.x) {
    const int r = q & 31, c = q >> 5;   // c: panel column
    li[r][c] = (ri + r < w.k && c < jb) ? w.L[(ri + r) + w.F * (j0 + c)] : T(0);
    lk[r][c] = (ck + r < w.k && c < jb) ? w.L[(ck + r) + w.F * (j0 + c)] : T(0);
  }
  if (threadIdx.x < jb) dv[threadIdx.x] = A.Dval[w.a + j0 + threadIdx.x];
  __syncthreads();
  for (int q = threadIdx.x; q < 32 * 32; q += blockDim.x) {
    const int r = q & 31, c = q >> 5;
    const int gr = ri + r, gc = ck + c;
    if (gr < w.k && gc < w.k && gr >= gc) {
      T acc = T(0);
      for (int t = 0; t < jb; ++t) acc += li[r][t] * (dv[t] * lk[c][t]);
      T* dst = w.L + gr + w.F * gc;
      *dst = *dst - acc;
    }
  }
}

// X[I, J] for the 32-row block I = blockIdx.y below J into buf (rows x 32 per
// front, row i - (j0 + jb) of the rest)
template <class T>
__global__ void __launch_bounds__(256) k_wide_inv(FrontArgs<T> A, const int32_t* fl, int j0, T* buf,
                                                  int64_t bstride) {
  const WideFront<T> w = wide_front(A, fl, blockIdx.x);
  if (j0 >= w.k) return;
  const int jb = min(kWideB, w.k - j0);
  const int t0 = j0 + jb;
  const int i0 = t0 + kWideB * (int)blockIdx.y;
  if (i0 >= w.k) return;
  __shared__ T bl[32][33], bx[32][33], xq[32][33], lq[32][33];
  for (int q = threadIdx.x; q < 32 * 32; q += blockDim.x) {
    const int r = q & 31, c = q >> 5;
    bl[r][c] = (r < jb && c < r) ? w.L[(j0 + r) + w.F * (j0 + c)] : T(0);
  }
  __syncthreads();
  unit_lower_inverse(bl, bx, jb);   // X_JJ
  // z[r][c] = L[i0 + r, j0 + c] + sum_{t0 <= q < i0 + r} X[i0 + r, q] L[q, j0 + c]
  const int r = threadIdx.x & 31, cg = threadIdx.x >> 5;   // row, columns cg, cg + 8, ...
  T z[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int c = cg + 8 * u;
    z[u] = (i0 + r < w.k && c < jb) ? w.L[(i0 + r) + w.F * (j0 + c)] : T(0);
  }
  for (int q0 = t0; q0 <= i0; q0 += kWideB) {
    __syncthreads();
    for (int q = threadIdx.x; q < 32 * 32; q += blockDim.x) {
      const int rr = q & 31, cc = q >> 5;
      // X[i0 + rr, q0 + cc]: strictly below the diagonal (the unit diagonal
      // is the L term above)
      const int gi = i0 + rr, gq = q0 + cc;
      xq[rr][cc] = (gi < w.k && gq < gi) ? w.L[gi + w.F * gq] : T(0);
      lq[rr][cc] = (q0 + rr < w.k && cc < jb) ? w.L[(q0 + rr) + w.F * (j0 + cc)] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int c = cg + 8 * u;
      T acc = z[u];
      for (int t = 0; t < 32; ++t) acc += xq[r][t] * lq[t][c];
      z[u] = acc;
    }
  }
  // out = -z X_JJ: out[r][c] = -sum_{t >= c} z[r][t] X_JJ[t][c]
  __syncthreads();
#pragma unroll
  for (int u = 0; u < 4; ++u) xq[r][cg + 8 * u] = z[u];
  __syncthreads();
  T* out = buf + (size_t)blockIdx.x * bstride;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int c = cg + 8 * u;
    if (i0 + r < w.k && c < jb) {
      T o = T(0);
      for (int t = c; t < jb; ++t) o += xq[r][t] * bx[t][c];
      out[(size_t)(i0 + r - t0) * 32 + c] = -o;
    }
  }
}

// The buffer into column block J below its diagonal block, X_JJ onto it.
template <class T>
__global__ void __launch_bounds__(256) k_wide_store(FrontArgs<T> A, const int32_t* fl, int j0,
                                                    const T* buf, int64_t bstride) {
  const WideFront<T> w = wide_front(A, fl, blockIdx.x);
  if (j0 >= w.k) return;
  const int jb = min(kWideB, w.k - j0);
  const int t0 = j0 + jb;
  const int i0 = t0 + kWideB * ((int)blockIdx.y - 1);   // block y = 0: the diagonal block
  const T* in = buf + (size_t)blockIdx.x * bstride;
  if (blockIdx.y == 0) {
    __shared__ T bl[32][33], bx[32][33];
    for (int q = threadIdx.x; q < 32 * 32; q += blockDim.x) {
      const int r = q & 31, c = q >> 5;
      bl[r][c] = (r < jb && c < r) ? w.L[(j0 + r) + w.F * (j0 + c)] : T(0);
    }
    __syncthreads();
    unit_lower_inverse(bl, bx, jb);
    for (int q = threadIdx.x; q < 32 * 32; q += blockDim.x) {
      const int r = q & 31, c = q >> 5;
      if (r < jb && c < r) w.L[(j0 + r) + w.F * (j0 + c)] = bx[r][c];
    }
    return;
  }
  if (i0 >= w.k) return;
  for (int q = threadIdx.x; q < 32 * 32; q += blockDim.x) {
    const int r = q >> 5, c = q & 31;
    if (i0 + r < w.k && c < jb) w.L[(i0 + r) + w.F * (j0 + c)] = in[(size_t)(i0 + r - t0) * 32 + c];
  }
}

// Row chunks of the update rows (items: front, first update row, rows <= 16):
// mode 0: L21 = F21 inv(L11)^T D^{-1}   (X[i, j] = D_j^{-1} sum_{c<=j} F21[i,c] inv(L11)[j,c])
// mode 1: W   = L21 inv(L11)            (W[i, j] = sum_{c>=j} L21[i,c] inv(L11)[c,j])
// in place: the chunk's outputs are staged in shared memory and written back
// after every read of the original rows.  32 x 32 tiles of inv(L11) and
// 16 x 32 tiles of the rows are staged in shared memory (coalesced loads).
template <class T>
__global__ void __launch_bounds__(256) k_panel_rows(FrontArgs<T> A, const int4* items, int item_begin,
                                                    int mode, T* gout, int kstride) {
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  // 16 x k, row-major: in shared memory, or (pivot blocks too wide for it)
  // in this item's slice of a global buffer
  T* out = gout ? gout + (size_t)blockIdx.x * 16 * (size_t)kstride : reinterpret_cast<T*>(dyn_smem);
  __shared__ T ta[16][33];            // rows x c
  __shared__ T tb[32][33];            // c x j  (or j x c)
  int4 it = items[item_begin + blockIdx.x];
  int s = it.x, r0 = it.y, nr = it.z;
  int a = A.sptr[s], k = A.sptr[s + 1] - a;
  int u = A.upd_ptr[s + 1] - A.upd_ptr[s];
  int64_t F = k + u;
  T* L = A.Lval + A.loff[s];
  T* R = L + k + r0;                  // first row of the chunk (column stride F)
  int tid = threadIdx.x;
  int orow = tid >> 4;                     // 0..15: output row
  int ocol = (tid & 15) * 2;               // two output columns within the j tile
  for (int j0 = 0; j0 < k; j0 += 32) {
    T acc0 = 0.0, acc1 = T(0);
    int cb = mode == 0 ? 0 : j0;           // inner range (triangle of inv(L11))
    int ce = mode == 0 ? min(k, j0 + 32) : k;
    for (int c0 = cb; c0 < ce; c0 += 32) {
      for (int q = tid; q < 16 * 32; q += 256) {
        int r = q & 15, c = q >> 4;
        ta[r][c] = (r < nr && c0 + c < k) ? R[r + F * (c0 + c)] : T(0);
      }
      for (int q = tid; q < 32 * 32; q += 256) {
        int x = q & 31, y = q >> 5;
        // mode 0 needs inv(L11)[j, c]: x = j offset (rows contiguous), y = c offset
        // mode 1 needs inv(L11)[c, j]: x = c offset (rows contiguous), y = j offset
        if (mode == 0)
          tb[y][x] = (j0 + x < k && c0 + y < k) ? L[(j0 + x) + F * (c0 + y)] : T(0);
        else
          tb[x][y] = (c0 + x < k && j0 + y < k) ? L[(c0 + x) + F * (j0 + y)] : T(0);
      }
      __syncthreads();
#pragma unroll 8
      for (int c = 0; c < 32; ++c) {
        T av = ta[orow][c];
        acc0 += av * tb[c][ocol];
        acc1 += av * tb[c][ocol + 1];
      }
      __syncthreads();
    }
    int j = j0 + ocol;
    if (mode == 0) {
      if (j < k) out[orow * k + j] = acc0 * A.Dinv[a + j];
      if (j + 1 < k) out[orow * k + j + 1] = acc1 * A.Dinv[a + j + 1];
    } else {
      if (j < k) out[orow * k + j] = acc0;
      if (j + 1 < k) out[orow * k + j + 1] = acc1;
    }
  }
  __syncthreads();
  for (int q = tid; q < nr * k; q += 256) {
    int r = q % nr, c = q / nr;
    R[r + F * c] = out[r * k + c];
  }
}

// Schur complement, one 32 x 32 tile (I >= J) of the update block per CTA:
// U[I, J] -= L21[I, :] D L21[J, :]^T, 32-column slabs staged in shared memory.
template <class T>
__global__ void __launch_bounds__(256) k_schur_tile(FrontArgs<T> A, const int4* items, int item_begin) {
  __shared__ T ta[32][33];
  __shared__ T tb[32][33];
  int4 it = items[item_begin + blockIdx.x];
  int s = it.x, I0 = it.y, J0 = it.z;
  int a = A.sptr[s], k = A.sptr[s + 1] - a;
  int u = A.upd_ptr[s + 1] - A.upd_ptr[s];
  int64_t F = k + u;
  const T* L21 = A.Lval + A.loff[s] + k;   // row i of L21 at L21[i + F c]
  T* U = A.Uval + A.uoff[s];
  int tid = threadIdx.x;
  int ty = tid >> 4, tx = tid & 15;              // 16 x 16 threads, 2 x 2 outputs each
  T c00 = 0.0, c01 = 0.0, c10 = 0.0, c11 = T(0);
  for (int c0 = 0; c0 < k; c0 += 32) {
    for (int q = tid; q < 32 * 32; q += 256) {
      int r = q & 31, c = q >> 5;
      bool okc = c0 + c < k;
      ta[r][c] = (I0 + r < u && okc) ? L21[(I0 + r) + F * (c0 + c)] : T(0);
      tb[r][c] = (J0 + r < u && okc) ? L21[(J0 + r) + F * (c0 + c)] * A.Dval[a + c0 + c] : T(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int c = 0; c < 32; ++c) {
      T a0 = ta[2 * ty][c], a1 = ta[2 * ty + 1][c];
      T b0 = tb[2 * tx][c], b1 = tb[2 * tx + 1][c];
      c00 += a0 * b0;
      c01 += a0 * b1;
      c10 += a1 * b0;
      c11 += a1 * b1;
    }
    __syncthreads();
  }
  int i = I0 + 2 * ty, j = J0 + 2 * tx;
  if (i < u && j < u) U[i + (int64_t)u * j] -= c00;
  if (i < u && j + 1 < u) U[i + (int64_t)u * (j + 1)] -= c01;
  if (i + 1 < u && j < u) U[(i + 1) + (int64_t)u * j] -= c10;
  if (i + 1 < u && j + 1 < u) U[(i + 1) + (int64_t)u * (j + 1)] -= c11;
}

// FB work item: 12 int32, loaded as three int4:
//   {front, first row/column, count <= 32, first pivot a,
//    k, u, gather base (forward) / upd_ptr (backward), upd_ptr (forward),
//    panel offset low, panel offset high, children's entries (forward), 0}
template <class T>
struct FBArgs {
  const int32_t* upd_idx;
  const int32_t* gptr;     // per front position: its children's update entries (CSR)
  const int32_t* gsrc;     // yvec slots of those entries, in child order
  const T* Lval;
  const T* Dinv;
  T* yvec;    // update vectors of the forward sweep (one per supernode)
  T* zbuf;    // forward result D^{-1} inv(L11) x of the pivot rows
  const int4* fwd_items;
  const int4* bwd_items;
};

template <class T>
FBArgs<T> fb_args(Problem& P);
template <>
FBArgs<double> fb_args<double>(Problem& P) {
  return FBArgs<double>{P.upd_idx.p, P.fb_gptr.p, P.fb_gsrc.p, P.Lval.p, P.Dinv.p, P.yvec.p,
                        P.zbuf.p, (const int4*)P.fwd_items.p, (const int4*)P.bwd_items.p};
}
template <>
FBArgs<zd> fb_args<zd>(Problem& P) {
  return FBArgs<zd>{P.upd_idx.p,      P.fb_gptr.p,     P.fb_gsrc.p,     zp(P.cx.Lval.p),
                    zp(P.cx.Dinv.p),  zp(P.cx.yvec.p), zp(P.cx.zbuf.p),
                    (const int4*)P.fwd_items.p, (const int4*)P.bwd_items.p};
}
template <>
FBArgs<float> fb_args<float>(Problem& P) {
  return FBArgs<float>{P.upd_idx.p, P.fb_gptr.p, P.fb_gsrc.p, P.Lval32.p, P.Dinv32.p, P.yvec32.p,
                       P.zbuf32.p, (const int4*)P.fwd_items.p, (const int4*)P.bwd_items.p};
}

// Children's update entries of one front position, gathered in list
// (child) order onto acc: the list is [g0, g1) of gsrc, and its first two
// source indices sa, sb (-1 past the end) are static, so callers load them
// before they wait for the vectors; then both values load together.
struct GatherPos {
  int g0, g1, sa, sb;
};
template <class T>
__device__ __forceinline__ GatherPos gather_plan(const FBArgs<T>& A, int gpos) {
  GatherPos q;
  q.g0 = A.gptr[gpos];
  q.g1 = A.gptr[gpos + 1];
  q.sa = q.g0 < q.g1 ? A.gsrc[q.g0] : -1;
  q.sb = q.g0 + 1 < q.g1 ? A.gsrc[q.g0 + 1] : -1;
  return q;
}
template <class T>
__device__ __forceinline__ T gather_sum(const FBArgs<T>& A, T acc, const GatherPos& q) {
  const T va = q.sa >= 0 ? __ldcg(A.yvec + q.sa) : T(0);
  const T vb = q.sb >= 0 ? __ldcg(A.yvec + q.sb) : T(0);
  if (q.sa >= 0) acc += va;
  if (q.sb >= 0) acc += vb;
  for (int g = q.g0 + 2; g < q.g1; ++g) acc += __ldcg(A.yvec + A.gsrc[g]);
  return acc;
}

// Adds v[t] x[t] for t < nt (nt warp-uniform, at most 8; x in shared
// memory, read only below nt) to the warp's partial sums.  In FP64 the
// products past nt are not issued, since each FP64 warp instruction holds
// the SM sub-partition's FP64 pipe for 64 cycles whatever its lanes do, and
// one accumulator suffices, since a dependent FP64 FMA waits no longer than
// that issue interval.  Other types keep four accumulators and zero weights.
template <class T>
__device__ __forceinline__ void chunk_acc(T (&s)[4], const T* v, const T* x, int nt) {
  if constexpr (std::is_same<T, double>::value) {
    double a = s[0];
    if (nt >= 8) {
#pragma unroll
      for (int t = 0; t < 8; ++t) a = fma(v[t], x[t], a);
    } else {
      switch (nt) {
        case 7: a = fma(v[6], x[6], a); [[fallthrough]];
        case 6: a = fma(v[5], x[5], a); [[fallthrough]];
        case 5: a = fma(v[4], x[4], a); [[fallthrough]];
        case 4: a = fma(v[3], x[3], a); [[fallthrough]];
        case 3: a = fma(v[2], x[2], a); [[fallthrough]];
        case 2: a = fma(v[1], x[1], a); [[fallthrough]];
        case 1: a = fma(v[0], x[0], a); [[fallthrough]];
        default: break;
      }
    }
    s[0] = a;
  } else {
    T w[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) w[t] = t < nt ? x[t] : T(0);
    s[0] += v[0] * w[0];
    s[1] += v[1] * w[1];
    s[2] += v[2] * w[2];
    s[3] += v[3] * w[3];
    s[0] += v[4] * w[4];
    s[1] += v[5] * w[5];
    s[2] += v[6] * w[6];
    s[3] += v[7] * w[7];
  }
}
template <class T>
__device__ __forceinline__ T chunk_total(const T (&s)[4]) {
  if constexpr (std::is_same<T, double>::value)
    return s[0];
  else
    return (s[0] + s[1]) + (s[2] + s[3]);
}

// Forward sweep, one work item = up to 32 RC consecutive rows of one front's
// panel P = [inv(L11); W], W = L21 inv(L11):
//   xg  = x_s + (children's update vectors at the pivot rows)
//   z   = inv(L11) xg           -> zbuf = D^{-1} z   (pivot rows)
//   y_s = (children at the update rows) - W xg      (update rows)
// Lanes run down the rows (coalesced columns).  Warp w takes row chunk
// w mod RC (32 rows) and column part w / RC of 8 / RC, keeping eight loads in
// flight; pivot rows only use the columns up to the chunk's last row.  RC = 1
// for long panels (all eight warps split the columns of 32 rows), RC = 4 for
// the short ones at the bottom of the tree (one item covers a small front and
// its gather is done once).  Vectors written by other work items (update
// vectors, right-hand side) are read through L2 (__ldcg).
template <class T, int RC>
__device__ __forceinline__ void fb_fwd_item(const FBArgs<T>& A, int item, const T* xin,
                                            T* xg) {
  constexpr int NP = 8 / RC;          // column parts per row chunk
  __shared__ T part[8][32];
  __shared__ T yadd[32 * RC];
  const int4* ip = A.fwd_items + 3 * (int64_t)item;
  int4 i0 = ip[0], i1 = ip[1], i2 = ip[2];
  int r0 = i0.y, nr = i0.z, a = i0.w;
  int k = i1.x, u = i1.y, gbase = i1.z;
  int64_t F = k + u;
  const T* P = A.Lval + ((int64_t)(uint32_t)i2.x | ((int64_t)i2.y << 32));
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rc = warp % RC, cp = warp / RC;
  const int cr0 = r0 + 32 * rc;                       // first row of this warp's chunk
  const int cn = max(0, min(32, nr - 32 * rc));       // rows of the chunk
  int row = cr0 + min(lane, max(cn, 1) - 1);
  int cend = cr0 + cn <= k ? cr0 + cn : k;            // triangle: columns <= last pivot row
  if (cn == 0) cend = 0;
  int q = (cend + NP - 1) / NP;
  int cb = cp * q, ce = min(cend, cb + q);
  const T* pr = P + min(row, (int)F - 1);
  // Columns in chunks of eight with unconditional loads (clamped to a valid
  // column, weight zero past the warp's range) so that a chunk's loads are all
  // in flight together; the first chunk does not depend on the gathered
  // vector and is issued before the gather.
  const int cl = max(cend - 1, 0);
  T v[8];
#pragma unroll
  for (int t = 0; t < 8; ++t) v[t] = pr[F * min(cb + t, cl)];
  // the gather lists are static too: this thread's first pivot position and
  // its update row (if any) are planned before the wait
  const bool kids = i2.z != 0;   // the front has children's update entries
  const bool yrow = threadIdx.x < nr && r0 + (int)threadIdx.x >= k;
  GatherPos gp{0, 0, -1, -1}, gy{0, 0, -1, -1};
  if (kids && (int)threadIdx.x < k) gp = gather_plan(A, gbase + threadIdx.x);
  if (kids && yrow) gy = gather_plan(A, gbase + r0 + threadIdx.x);
  // this thread's pivot (if its row is one), needed after the reduction
  const T dinv = (int)threadIdx.x < nr && r0 + (int)threadIdx.x < k ? A.Dinv[a + r0 + threadIdx.x]
                                                                     : T(0);
  // the panels and item descriptors were written before this sweep; the
  // vectors below come from the previous kernels of the stream
  pdl_wait();
  // right-hand side plus the children's update vectors, summed per front
  // position in child order (deterministic, no write conflicts)
  if ((int)threadIdx.x < k) xg[threadIdx.x] = gather_sum(A, __ldcg(xin + a + threadIdx.x), gp);
  for (int t = threadIdx.x + blockDim.x; t < k; t += blockDim.x) {
    T acc = __ldcg(xin + a + t);
    if (kids) acc = gather_sum(A, acc, gather_plan(A, gbase + t));
    xg[t] = acc;
  }
  if (yrow) yadd[threadIdx.x] = gather_sum(A, T(0), gy);
  __syncthreads();
  T sacc[4] = {T(0), T(0), T(0), T(0)};
  for (int c = cb;;) {
    chunk_acc(sacc, v, xg + c, min(8, ce - c));
    c += 8;
    if (c >= ce) break;
#pragma unroll
    for (int t = 0; t < 8; ++t) v[t] = pr[F * min(c + t, cl)];
  }
  part[warp][lane] = chunk_total(sacc);
  __syncthreads();
  if (threadIdx.x < nr) {
    const int l = threadIdx.x;
    int i = r0 + l;
    const int lrc = l / 32, ll = l % 32;
    T dot = T(0);
#pragma unroll
    for (int pp = 0; pp < NP; ++pp) dot += part[pp * RC + lrc][ll];
    if (i < k) A.zbuf[a + i] = dot * dinv;
    else A.yvec[i1.w + (i - k)] = yadd[l] - dot;
  }
  __syncthreads();
}

template <class T, int RC>
__global__ void __launch_bounds__(256) k_fb_fwd(FBArgs<T> A, int item_begin, const T* xin) {
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  T* xg = reinterpret_cast<T*>(dyn_smem);
  fb_fwd_item<T, RC>(A, item_begin + blockIdx.x, xin, xg);
}

// Backward sweep, one work item = up to 32 pivot columns c of one front:
//   x_c = sum_{i >= c, i < k} inv(L11)[i, c] zbuf_i - sum_i W[i, c] x_struct(i)
// i.e. x_s = inv(L11)^T (D^{-1} z - L21^T x_struct) with W = L21 inv(L11).
// Each warp takes 32-row blocks of the item's columns: it loads the 32 x 32
// block with coalesced column reads (lanes down the rows) into shared
// memory, then each lane forms its own column's dot product from the staged
// block, so no lane-transpose reduction is needed; the warps' partial sums
// are added at the end in warp order.  Levels with few items (the top of the
// tree, long panels) use eight warps per item, the others four.  Optionally
// writes r_u = -x, r_l = sigma r_u + v_u.
// Operator outputs of the backward sweep from the solution entry x of
// Q x = y: real scalars r_u = -uscale x, r_l = -sigma x + v_u; complex shift
// s = sigma + i sigma_i (the real part of the complex operator):
// r_u = -Re x, r_l = Re(-s x) + v_u.
// The same with v_u[cc] already loaded (vuc; real factors only).
template <class T>
__device__ __forceinline__ void op_out_v(T sum, double sigma, double uscale,
                                         typename RealOf<T>::type vuc,
                                         typename RealOf<T>::type* ru, typename RealOf<T>::type* rl,
                                         int64_t cc) {
  using R = typename RealOf<T>::type;
  ru[cc] = (R)(uscale * (double)(-sum));
  rl[cc] = (R)(sigma * (double)(-sum)) + vuc;
}

template <class T>
__device__ __forceinline__ void op_out(T sum, double sigma, double sigma_i, double uscale,
                                       const typename RealOf<T>::type* vu,
                                       typename RealOf<T>::type* ru, typename RealOf<T>::type* rl,
                                       int64_t cc) {
  using R = typename RealOf<T>::type;
  if constexpr (std::is_same<T, zd>::value) {
    ru[cc] = -sum.re;
    rl[cc] = -(sigma * sum.re - sigma_i * sum.im) + vu[cc];
  } else {
    (void)sigma_i;
    ru[cc] = (R)(uscale * (double)(-sum));
    rl[cc] = (R)(sigma * (double)(-sum)) + vu[cc];
  }
}

// acc + sum_{t < nrow} trow[t] g[t] over a staged 32-row block of which
// the first nrow rows (warp-uniform) lie inside the front: the products of
// the rows past its end are zero and, in FP64, cost full issue slots.  R: the
// rows a lane covers in a full block (32, or 16 with two lanes per column).
template <class T, int R = 32>
__device__ __forceinline__ T block_acc(T acc, const T* trow, const T* g, int nrow) {
  if (nrow >= R) {
#pragma unroll
    for (int t = 0; t < R; ++t) acc += trow[t] * g[t];
  } else {
    for (int t = 0; t < nrow; ++t) acc += trow[t] * g[t];
  }
  return acc;
}

template <class T>
__device__ __forceinline__ T shfl_down_t(T v, int d) {
  return __shfl_down_sync(0xffffffffu, v, d);
}

template <class T, int NW>
__device__ __forceinline__ void fb_bwd_item(const FBArgs<T>& A, int item, T* x, double sigma,
                                            const typename RealOf<T>::type* vu,
                                            typename RealOf<T>::type* ru,
                                            typename RealOf<T>::type* rl,
                                            T* smem, double uscale, double sigma_i) {
  T(*tile)[32][33] = reinterpret_cast<T(*)[32][33]>(smem);
  __shared__ T gs[NW][32];
  __shared__ T red[NW][32];
  const int4* ip = A.bwd_items + 3 * (int64_t)item;
  int4 i0 = ip[0], i1 = ip[1], i2 = ip[2];
  int c0 = i0.y, nc = i0.z, a = i0.w;
  int k = i1.x, u = i1.y;
  int64_t F = k + u;
  const T* P = A.Lval + ((int64_t)(uint32_t)i2.x | ((int64_t)i2.y << 32)) + F * c0;
  const int32_t* st = A.upd_idx + i1.z;
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T acc = T(0);
  // the first block's panel entries were written before this sweep: load them
  // before waiting for the previous kernels (zbuf and x come from those)
  T v[32];
  int xi0 = -1;   // first block: solution index of an update row (static)
  {
    const int64_t i = c0 + 32 * warp + lane;
    const T* pr = P + (i < F ? i : F - 1);
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = pr[F * min(q, nc - 1)];
    if (i < F && i >= k) xi0 = st[i - k];
  }
  pdl_wait();
  // this thread's entry of v_u, for r_l after the reduction
  typename RealOf<T>::type vuc = 0;
  if (ru && (int)threadIdx.x < nc) vuc = vu[a + c0 + threadIdx.x];
  bool first = true;
  for (int64_t r0 = c0 + 32 * warp; r0 < F; r0 += 32 * NW) {
    int64_t i = r0 + lane;
    int64_t ic = i < F ? i : F - 1;
    T g = T(0);
    if (i < F) g = i < k ? __ldcg(A.zbuf + a + i) : -__ldcg(x + (first ? xi0 : st[i - k]));
    const T* pr = P + ic;
    if (!first) {
#pragma unroll
      for (int q = 0; q < 32; ++q) v[q] = pr[F * min(q, nc - 1)];
    }
    first = false;
    gs[warp][lane] = g;
#pragma unroll
    for (int q = 0; q < 32; ++q) tile[warp][q][lane] = v[q];
    __syncwarp();
    acc = block_acc(acc, tile[warp][lane], gs[warp], (int)min((int64_t)32, F - r0));
    __syncwarp();
  }
  red[warp][lane] = acc;
  __syncthreads();
  if (threadIdx.x < nc) {
    const int l = threadIdx.x;
    T sum = T(0);
#pragma unroll
    for (int w = 0; w < NW; ++w) sum += red[w][l];
    int cc = a + c0 + l;
    x[cc] = sum;
    if constexpr (std::is_same<T, zd>::value) {
      if (ru) op_out<T>(sum, sigma, sigma_i, uscale, vu, ru, rl, cc);
    } else {
      if (ru) op_out_v<T>(sum, sigma, uscale, vuc, ru, rl, cc);
    }
  }
  __syncthreads();
}

template <class T, int NW>
__global__ void __launch_bounds__(NW * 32, NW == 4 ? 4 : 1)
    k_fb_bwd(FBArgs<T> A, int item_begin, T* x, double sigma,
             const typename RealOf<T>::type* vu, typename RealOf<T>::type* ru,
             typename RealOf<T>::type* rl, double uscale, double sigma_i) {
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  T* bwd_smem = reinterpret_cast<T*>(dyn_smem);
  fb_bwd_item<T, NW>(A, item_begin + blockIdx.x, x, sigma, vu, ru, rl, bwd_smem, uscale, sigma_i);
}

// ---- dependency-driven sweeps of the upper tree levels ----
//
// Above the leaves each level has few items and the level-by-level launches
// leave most of the GPU idle while a level's few items run their latency
// chains.  These two kernels run all levels from `first level` upwards
// (forward) or downwards (backward) in one launch: a block takes the next
// item by ticket (atomic counter; items are ordered so that every item
// depends only on items with smaller tickets), waits until the fronts it
// depends on are complete, runs the item and marks it complete.  A block
// only ever waits for smaller tickets, which running blocks hold, so the
// launch cannot deadlock whatever the number of resident blocks.
//
// Completion counters are cumulative over solves (epoch e = number of this
// handle's sweeps so far): forward, kdone[s] counts the finished items of
// the children of s inside the launch, complete when it reaches
// e * kid_items[s]; backward, bdone[s] counts the finished items of s,
// complete at e * bwd_items[s].  Producers publish with a release fence and
// an atomic add; one thread of the consumer polls with an acquire load
// (bounded: a wait that runs out records a timeout in the status word and
// the item runs on stale data; the host reports the error) and the block
// synchronises before reading.  The last block of a launch resets the
// ticket counters for the next launch.
struct FBDep {
  const int32_t* parent;     // supernode parent (-1: root)
  const int32_t* kid_items;  // forward: items of the children inside the launch
  const int32_t* bwd_items;  // backward items of each supernode
  unsigned* kdone;           // cumulative counters (see above)
  unsigned* bdone;
  unsigned* ticket;          // [0] ticket, [1] blocks finished
  unsigned epoch;
  DevStatus* status;
};

constexpr uint32_t kDepWaitLimit = 1u << 24;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// thread 0: wait until *cnt reaches target (modular comparison)
__device__ __forceinline__ void dep_wait(const unsigned* cnt, unsigned target, DevStatus* st) {
  uint32_t it = 0;
  while ((int)(ld_acquire_u32(cnt) - target) < 0) {
    if (++it >= kDepWaitLimit) {
      atomicCAS(&st->timeout, 0, 2);
      return;
    }
  }
}

// one release add (the item's writes, ordered before it by the preceding
// block barrier, are visible to whoever acquires the counter)
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int dep_ticket(unsigned* ticket) {
  __shared__ int tk;
  __syncthreads();
  if (threadIdx.x == 0) tk = (int)atomicAdd(ticket, 1u);
  __syncthreads();
  return tk;
}

__device__ __forceinline__ void dep_finish_launch(unsigned* ticket) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(ticket + 1, 1u) == gridDim.x - 1) {   // last block: reset for the next launch
      atomicExch(ticket, 0u);
      atomicExch(ticket + 1, 0u);
      __threadfence();
    }
  }
}

// Forward item of the dependency-driven sweep.  Same arithmetic as
// fb_fwd_item; everything that does not depend on the children (up to
// kPreChunks chunks of eight panel columns per warp, the right-hand side and
// the gather indices) is loaded before the block waits for the children, so
// that only the children's update values are read after the wait.
constexpr int kPreChunks = 5;
constexpr int kBwdHalfRows = 192;   // fronts whose backward items take at most 16 columns

template <class T, int RC>
__device__ __forceinline__ void fb_fwd_item_pre(const FBArgs<T>& A, const FBDep& D, int item,
                                                const T* xin, T* xg) {
  constexpr int NP = 8 / RC;
  __shared__ T part[8][32];
  __shared__ T yadd[32 * RC];
  const int4* ip = A.fwd_items + 3 * (int64_t)item;
  int4 i0 = ip[0], i1 = ip[1], i2 = ip[2];
  const int s = i0.x, r0 = i0.y, nr = i0.z, a = i0.w;
  const int k = i1.x, u = i1.y, gbase = i1.z;
  const int64_t F = k + u;
  const T* P = A.Lval + ((int64_t)(uint32_t)i2.x | ((int64_t)i2.y << 32));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rc = warp % RC, cp = warp / RC;
  const int cr0 = r0 + 32 * rc;
  const int cn = max(0, min(32, nr - 32 * rc));
  const int row = cr0 + min(lane, max(cn, 1) - 1);
  int cend = cr0 + cn <= k ? cr0 + cn : k;
  if (cn == 0) cend = 0;
  const int q = (cend + NP - 1) / NP;
  const int cb = cp * q, ce = min(cend, cb + q);
  const T* pr = P + min(row, (int)F - 1);
  const int cl = max(cend - 1, 0);
  T v[kPreChunks][8];
#pragma unroll
  for (int c = 0; c < kPreChunks; ++c)
#pragma unroll
    for (int t = 0; t < 8; ++t) v[c][t] = pr[F * min(cb + 8 * c + t, cl)];
  const bool kids = i2.z != 0;
  // this thread's gather positions (at most two before the wait): the
  // right-hand side and the first two source indices of each list
  T xr[2];
  GatherPos gp[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int t = threadIdx.x + 256 * h;
    xr[h] = T(0);
    gp[h] = GatherPos{0, 0, -1, -1};
    if (t < k) {
      xr[h] = __ldcg(xin + a + t);
      if (kids) gp[h] = gather_plan(A, gbase + t);
    }
  }
  const bool yrow = threadIdx.x < nr && r0 + (int)threadIdx.x >= k;
  GatherPos gy{0, 0, -1, -1};
  if (yrow && kids) gy = gather_plan(A, gbase + r0 + threadIdx.x);
  const T dinv = (int)threadIdx.x < nr && r0 + (int)threadIdx.x < k ? A.Dinv[a + r0 + threadIdx.x]
                                                                     : T(0);
  // the children's update vectors are complete
  if (threadIdx.x == 0) dep_wait(D.kdone + s, D.epoch * (unsigned)D.kid_items[s], D.status);
  __syncthreads();
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int t = threadIdx.x + 256 * h;
    if (t < k) xg[t] = gather_sum(A, xr[h], gp[h]);
  }
  for (int t = threadIdx.x + 512; t < k; t += blockDim.x) {
    T acc = __ldcg(xin + a + t);
    if (kids) acc = gather_sum(A, acc, gather_plan(A, gbase + t));
    xg[t] = acc;
  }
  if (yrow) yadd[threadIdx.x] = gather_sum(A, T(0), gy);
  __syncthreads();
  T sacc[4] = {T(0), T(0), T(0), T(0)};
  int c = cb;
#pragma unroll
  for (int ch = 0; ch < kPreChunks; ++ch) {
    if (c < ce) chunk_acc(sacc, v[ch], xg + c, min(8, ce - c));
    c += 8;
  }
  for (; c < ce; c += 8) {   // columns beyond the preloaded chunks (largest fronts only)
    T vv[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) vv[t] = pr[F * min(c + t, cl)];
    chunk_acc(sacc, vv, xg + c, min(8, ce - c));
  }
  part[warp][lane] = chunk_total(sacc);
  __syncthreads();
  if (threadIdx.x < nr) {
    const int l = threadIdx.x;
    const int i = r0 + l;
    const int lrc = l / 32, ll = l % 32;
    T dot = T(0);
#pragma unroll
    for (int pp = 0; pp < NP; ++pp) dot += part[pp * RC + lrc][ll];
    if (i < k) A.zbuf[a + i] = dot * dinv;
    else A.yvec[i1.w + (i - k)] = yadd[l] - dot;
  }
  __syncthreads();
}

// Backward item of the dependency-driven sweep.  Same arithmetic as
// fb_bwd_item with eight warps; the panel blocks (up to two per warp), the
// pivot-row values of the forward sweep and the indices of the update rows
// are loaded before the block waits for its parent; only the solution
// entries of the ancestors are read after the wait.  NC = 32: lane c forms
// column c's dot product over the 32 rows of a staged block.  NC = 16 (items
// of at most 16 columns, made for the wide fronts at the top of the tree,
// whose items are bound by their own FP64 issue): lanes c and c + 16 each
// take half of the block's rows of column c, so every FP64 instruction still
// does 32 products and an item costs half the instructions; the two halves
// meet in one shuffle at the end.
template <class T, int NC>
__device__ __forceinline__ void fb_bwd_item_pre(const FBArgs<T>& A, const FBDep& D, int item, T* x,
                                                double sigma, const typename RealOf<T>::type* vu,
                                                typename RealOf<T>::type* ru,
                                                typename RealOf<T>::type* rl, T* smem,
                                                double uscale) {
  constexpr int NW = 8;
  T(*tile)[32][33] = reinterpret_cast<T(*)[32][33]>(smem);
  __shared__ T gs[NW][32];
  __shared__ T red[NW][32];
  const int4* ip = A.bwd_items + 3 * (int64_t)item;
  int4 i0 = ip[0], i1 = ip[1], i2 = ip[2];
  const int s = i0.x, c0 = i0.y, nc = i0.z, a = i0.w;
  const int k = i1.x, u = i1.y;
  const int64_t F = k + u;
  const T* P = A.Lval + ((int64_t)(uint32_t)i2.x | ((int64_t)i2.y << 32)) + F * c0;
  const int32_t* st = A.upd_idx + i1.z;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // this lane's column and first row of a staged block when computing
  const int ccol = NC == 32 ? lane : (lane & 15);
  const int hrow = NC == 32 ? 0 : 16 * (lane >> 4);
  // blocks 0 and 1 of this warp: rows c0 + 32 warp + lane + 256 b
  T v[2][NC];
  T zv[2];
  int xi[2];   // update rows: index into x (-1: pivot row or past the front)
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    const int64_t i = c0 + 32 * warp + lane + 32 * NW * b;
    const T* pr = P + (i < F ? i : F - 1);
#pragma unroll
    for (int q = 0; q < NC; ++q) v[b][q] = pr[F * min(q, nc - 1)];
    zv[b] = T(0);
    xi[b] = -1;
    if (i < F) {
      if (i < k) zv[b] = __ldcg(A.zbuf + a + i);
      else xi[b] = st[i - k];
    }
  }
  // this thread's entry of v_u (written before the launch), for r_l
  typename RealOf<T>::type vuc = 0;
  if (ru && (int)threadIdx.x < nc) vuc = vu[a + c0 + threadIdx.x];
  const int pa = D.parent[s];
  if (threadIdx.x == 0 && pa >= 0)
    dep_wait(D.bdone + pa, D.epoch * (unsigned)D.bwd_items[pa], D.status);
  __syncthreads();
  T acc = T(0);
  // rows of a staged block at rb inside the front, counted from this lane's
  // first row (the products of the rows past the end are zero and, in FP64,
  // cost full issue slots)
  auto nrows = [&](int64_t rb) {
    return (int)max((int64_t)0, min((int64_t)(NC == 32 ? 32 : 16), F - rb - hrow));
  };
  // blocks 0 and 1 from the preloaded registers (compile-time indices), the
  // rest streamed
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    const int64_t rb = c0 + 32 * warp + 32 * NW * b;
    if (rb < F) {
      gs[warp][lane] = xi[b] >= 0 ? -__ldcg(x + xi[b]) : zv[b];
#pragma unroll
      for (int q = 0; q < NC; ++q) tile[warp][q][lane] = v[b][q];
      __syncwarp();
      acc = block_acc<T, NC == 32 ? 32 : 16>(acc, tile[warp][ccol] + hrow, gs[warp] + hrow, nrows(rb));
      __syncwarp();
    }
  }
  for (int64_t r0 = c0 + 32 * warp + 2 * 32 * NW; r0 < F; r0 += 32 * NW) {
    const int64_t i = r0 + lane;
    T g = T(0);
    if (i < F) g = i < k ? __ldcg(A.zbuf + a + i) : -__ldcg(x + st[i - k]);
    const T* pr = P + (i < F ? i : F - 1);
#pragma unroll
    for (int q = 0; q < NC; ++q) tile[warp][q][lane] = pr[F * min(q, nc - 1)];
    gs[warp][lane] = g;
    __syncwarp();
    acc = block_acc<T, NC == 32 ? 32 : 16>(acc, tile[warp][ccol] + hrow, gs[warp] + hrow, nrows(r0));
    __syncwarp();
  }
  if constexpr (NC == 16) acc += shfl_down_t(acc, 16);
  red[warp][lane] = acc;
  __syncthreads();
  if (threadIdx.x < nc) {
    const int l = threadIdx.x;
    T sum = T(0);
#pragma unroll
    for (int w = 0; w < NW; ++w) sum += red[w][l];
    const int cc = a + c0 + l;
    x[cc] = sum;
    if (ru) op_out_v<T>(sum, sigma, uscale, vuc, ru, rl, cc);
  }
  __syncthreads();
}

template <class T>
__global__ void __launch_bounds__(256) k_fb_fwd_dep(FBArgs<T> A, FBDep D, int item_begin,
                                                    int n_items, const T* xin) {
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  T* xg = reinterpret_cast<T*>(dyn_smem);
  pdl_wait();
  for (;;) {
    const int t = dep_ticket(D.ticket);
    if (t >= n_items) break;
    const int item = item_begin + t;
    const int s = A.fwd_items[3 * (int64_t)item].x;
    if (A.fwd_items[3 * (int64_t)item + 2].w == 4) fb_fwd_item_pre<T, 4>(A, D, item, xin, xg);
    else fb_fwd_item_pre<T, 1>(A, D, item, xin, xg);
    if (threadIdx.x == 0) {   // the item's outputs are written (the item ends in a barrier)
      const int pa = D.parent[s];
      if (pa >= 0) red_release_add(D.kdone + pa, 1u);
    }
  }
  dep_finish_launch(D.ticket);
}

template <class T>
__global__ void __launch_bounds__(256, 1) k_fb_bwd_dep(FBArgs<T> A, FBDep D, const int32_t* order,
                                                    int n_items, T* x, double sigma, const T* vu,
                                                    T* ru, T* rl, double uscale) {
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  T* smem = reinterpret_cast<T*>(dyn_smem);
  pdl_wait();
  for (;;) {
    const int t = dep_ticket(D.ticket);
    if (t >= n_items) break;
    const int item = order[t];
    const int s = A.bwd_items[3 * (int64_t)item].x;
    if (A.bwd_items[3 * (int64_t)item].z <= 16)
      fb_bwd_item_pre<T, 16>(A, D, item, x, sigma, vu, ru, rl, smem, uscale);
    else
      fb_bwd_item_pre<T, 32>(A, D, item, x, sigma, vu, ru, rl, smem, uscale);
    if (threadIdx.x == 0) red_release_add(D.bdone + s, 1u);
  }
  dep_finish_launch(D.ticket);
}

// refinement helpers (FP64 vectors, FP32 correction)
__global__ void k_to_f32(const double* a, float* b, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

__global__ void k_ir_accum(double* x, const float* d, int64_t n, int first) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) x[i] = first ? (double)d[i] : x[i] + (double)d[i];
}

// r = y - (s2 M + s1 C + K) x in the ND order, 8 lanes per row; the FP32 copy
// (next correction's right-hand side) or the FP64 residual
template <class R>
__device__ __forceinline__ void ir_residual_row(const int32_t* rowptr, const int32_t* col,
                                                const double* K, const double* M, const double* C,
                                                double s2, double s1, const double* x,
                                                const double* y, R* r, int64_t N) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t row = t / 8;
  int sub = t % 8;
  double acc = 0.0;
  if (row < N)
    for (int32_t q = rowptr[row] + sub; q < rowptr[row + 1]; q += 8)
      acc += (s2 * M[q] + s1 * C[q] + K[q]) * x[col[q]];
  for (int o = 4; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, 8);
  if (row < N && sub == 0) r[row] = (R)(y[row] - acc);
}

__global__ void k_ir_residual(const int32_t* rowptr, const int32_t* col, const double* K,
                              const double* M, const double* C, double s2, double s1,
                              const double* x, const double* y, float* r, int64_t N) {
  ir_residual_row<float>(rowptr, col, K, M, C, s2, s1, x, y, r, N);
}

__global__ void k_ir_residual64(const int32_t* rowptr, const int32_t* col, const double* K,
                                const double* M, const double* C, double s2, double s1,
                                const double* x, const double* y, double* r, int64_t N) {
  ir_residual_row<double>(rowptr, col, K, M, C, s2, s1, x, y, r, N);
}

// operator outputs from the solution x of Q x = y: r_u = -x, r_l = s r_u + v_u
__global__ void k_op_out(const double* x, double s, const double* vu, double* ru, double* rl,
                         int64_t n, double uscale) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) {
    double v = -x[i];
    ru[i] = uscale * v;
    rl[i] = s * v + vu[i];
  }
}

// seeded right-hand side in [-0.5, 0.5) (splitmix64 of seed + i)
__global__ void k_probe_rhs(uint64_t seed, double* v, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t z = seed + (uint64_t)i + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  v[i] = (double)(z >> 11) * 0x1.0p-53 - 0.5;
}

__global__ void k_gather(const int32_t* idx, const double* src, double* dst, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[idx[i]];
}

__global__ void k_gather2(const int32_t* idx, const double2* src, double2* dst, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[idx[i]];
}

__global__ void k_scatter2(const int32_t* idx, const double2* src, double2* dst, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) dst[idx[i]] = src[i];
}

__global__ void k_scatter(const int32_t* idx, const double* src, double* dst, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) dst[idx[i]] = src[i];
}

}  // namespace

// tree levels below this one run as one launch per level and sweep (the
// leaves stream the bulk of the factor); the levels from it up run in the
// dependency-driven launches
constexpr int kDepLevel = 3;

template <class T>
constexpr size_t bwd_smem(int nw) {
  return sizeof(T) * (size_t)nw * 32 * 33;
}

void factor_configure(size_t smem_max) {
  smem_at_least((const void*)k_fb_bwd<double, 8>, bwd_smem<double>(8));
  smem_at_least((const void*)k_fb_bwd<float, 8>, bwd_smem<float>(8));
  smem_at_least((const void*)k_fb_bwd_dep<double>, bwd_smem<double>(8));
  smem_at_least((const void*)k_fb_bwd_dep<float>, bwd_smem<float>(8));
  if (smem_max > 48 * 1024) {
    smem_at_least((const void*)k_fb_fwd<double, 1>, smem_max);
    smem_at_least((const void*)k_fb_fwd<float, 1>, smem_max / 2);
    smem_at_least((const void*)k_fb_fwd<double, 4>, smem_max);
    smem_at_least((const void*)k_fb_fwd<float, 4>, smem_max / 2);
  }
}

// largest dynamic shared memory of a forward sweep item in FP64 (the
// gathered right-hand side of the largest pivot block)
size_t smem_fwd_max(const Problem& P) {
  int k = 1;
  for (int v : P.lvl_maxK) k = std::max(k, v);
  return sizeof(double) * (size_t)k;
}

void factor_plan(Problem& P) {
  Plan& L = P.plan;
  std::vector<int32_t> rows, tiles;
  P.row_lvl.assign(L.nlevels + 1, 0);
  P.tile_lvl.assign(L.nlevels + 1, 0);
  for (int l = 0; l < L.nlevels; ++l) {
    for (int q = L.lvl_ptr[l]; q < L.lvl_ptr[l + 1]; ++q) {
      int s = L.lvl_nodes[q];
      int u = L.upd_ptr[s + 1] - L.upd_ptr[s];
      for (int r = 0; r < u; r += 16) rows.insert(rows.end(), {s, r, std::min(16, u - r), 0});
      for (int I = 0; I < u; I += 32)
        for (int J = 0; J <= I; J += 32) tiles.insert(tiles.end(), {s, I, J, 0});
    }
    P.row_lvl[l + 1] = (int32_t)(rows.size() / 4);
    P.tile_lvl[l + 1] = (int32_t)(tiles.size() / 4);
  }
  P.row_items.upload(rows, P.stream);
  P.tile_items.upload(tiles, P.stream);
  // pivot blocks of each level: small ones one CTA each, large ones a
  // cluster, wider ones by the blocked multi-CTA kernels (k_wide_*); the
  // complex factor's cluster panel holds twice the bytes, so its blocks of
  // more than kClusterMaxKc pivots are wide
  int wide_fronts = 0, wide_k = 0;
  auto classify = [&](int kmax_cluster, std::vector<int32_t>& lv) {
    std::vector<int32_t> out;
    lv.assign(3 * L.nlevels + 1, 0);
    for (int l = 0; l < L.nlevels; ++l)
      for (int cls = 0; cls < 3; ++cls) {
        int n = 0;
        for (int q = L.lvl_ptr[l]; q < L.lvl_ptr[l + 1]; ++q) {
          int sn = L.lvl_nodes[q];
          int k = L.sptr[sn + 1] - L.sptr[sn];
          const int c = k < kClusterMinK ? 0 : (k <= std::min(kmax_cluster, kWideFromK) ? 1 : 2);
          if (c == cls) {
            out.push_back(sn);
            ++n;
            if (cls == 2) wide_k = std::max(wide_k, k);
          }
        }
        if (cls == 2) wide_fronts = std::max(wide_fronts, n);
        lv[3 * l + cls + 1] = (int32_t)out.size();
      }
    return out;
  };
  P.piv_fronts.upload(classify(kClusterMaxK, P.piv_lvl), P.stream);
  P.cx.piv_fronts.upload(classify(kClusterMaxKc, P.cx.piv_lvl), P.stream);
  // wide pivot blocks: X_JJ (32 x 32) and a rows x 32 buffer per front, in
  // doubles for 16-byte scalars
  P.wide_bstride = 32 * (int64_t)std::max(wide_k, 1);
  if (wide_fronts > 0)
    P.wide_scratch.alloc((size_t)wide_fronts * (32 * 32 + (size_t)P.wide_bstride) * 2);
  {
    size_t cs = sizeof(double) * 32 * (size_t)kClusterMaxK;
    smem_at_least((const void*)k_pivot_cluster<double>, cs);
    smem_at_least((const void*)k_pivot_cluster<float>, cs / 2);
    smem_at_least((const void*)k_pivot_cluster<zd>, sizeof(zd) * 32 * (size_t)kClusterMaxKc);
  }
  P.Dval.alloc(L.N);
  // row panels: 16 x k per item in shared memory, else a global buffer for
  // the levels whose pivot blocks are wider (sized for 16-byte scalars)
  const size_t kpan = smem_fwd_max(P) / sizeof(double);
  size_t smem = std::min(sizeof(double) * 16 * kpan, kPanelSmemMax);
  if (smem > 48 * 1024) smem_at_least((const void*)k_panel_rows<double>, smem);
  if (smem / 2 > 48 * 1024) smem_at_least((const void*)k_panel_rows<float>, smem / 2);
  {
    size_t need = 0;
    for (int l = 0; l < L.nlevels; ++l)
      if (sizeof(zd) * 16 * (size_t)P.lvl_maxK[l] > kPanelSmemMax)   // the widest scalar
        need = std::max(need, (size_t)(P.row_lvl[l + 1] - P.row_lvl[l]) * 16 *
                                  (size_t)P.lvl_maxK[l] * 2);
    if (need > 0) P.panel_scratch.alloc(need);
  }
  size_t piv = sizeof(double) * (size_t)L.max_front;
  if (piv > 48 * 1024) smem_at_least((const void*)k_pivot_factor<double>, piv);
  if (piv / 2 > 48 * 1024) smem_at_least((const void*)k_pivot_factor<float>, piv / 2);
  // the complex kernels' row panels and pivot staging hold k complex values
  // per row (k = the largest pivot block)
  const size_t kmax = smem_fwd_max(P) / sizeof(double);
  const size_t zrows = sizeof(zd) * 16 * kmax, zpiv = sizeof(zd) * kmax;
  if (zrows > 48 * 1024)
    smem_at_least((const void*)k_panel_rows<zd>, std::min(zrows, kPanelSmemMax));
  if (zpiv > 48 * 1024 && zpiv <= kSmemOptIn) smem_at_least((const void*)k_pivot_factor<zd>, zpiv);
  smem_at_least((const void*)k_fb_bwd<zd, 8>, bwd_smem<zd>(8));
  if (2 * smem_fwd_max(P) > 48 * 1024)
    smem_at_least((const void*)k_fb_fwd<zd, 1>, 2 * smem_fwd_max(P));
  if (2 * smem_fwd_max(P) > 48 * 1024)
    smem_at_least((const void*)k_fb_fwd<zd, 4>, 2 * smem_fwd_max(P));
}

// tc: the products after the pivot blocks (L21, the Schur update, W) run on
// the tensor cores (tcfront.cu) instead of k_panel_rows / k_schur_tile
// The wide pivot blocks of level l (the k_wide_* steps, every front of the
// level in each launch).
template <class T>
void launch_wide_pivots(Problem& P, const FrontArgs<T>& A, const int32_t* fl, int nwide, int l) {
  cudaStream_t s = P.stream;
  const int kmax = P.lvl_maxK[l];
  const int nb = (kmax + kWideB - 1) / kWideB;
  T* xjj = reinterpret_cast<T*>(P.wide_scratch.p);
  T* buf = xjj + (size_t)nwide * 32 * 32;
  for (int J = 0; J < nb; ++J) {
    const int j0 = J * kWideB;
    const int nrb = nb - J - 1;   // 32-row blocks below J (largest front)
    k_wide_diag<T><<<nwide, 256, 0, s>>>(A, fl, j0, xjj);
    RQ_CUDA(cudaGetLastError());
    if (nrb > 0) {
      k_wide_panel<T><<<dim3(nwide, nrb), 256, 0, s>>>(A, fl, j0, xjj);
      RQ_CUDA(cudaGetLastError());
      k_wide_update<T><<<dim3(nwide, nrb * (nrb + 1) / 2), 256, 0, s>>>(A, fl, j0);
      RQ_CUDA(cudaGetLastError());
    }
    P.launches += nrb > 0 ? 3 : 1;
  }
  for (int J = nb - 1; J >= 0; --J) {
    const int j0 = J * kWideB;
    const int nrb = nb - J - 1;
    if (nrb > 0) {
      k_wide_inv<T><<<dim3(nwide, nrb), 256, 0, s>>>(A, fl, j0, buf, P.wide_bstride);
      RQ_CUDA(cudaGetLastError());
    }
    k_wide_store<T><<<dim3(nwide, nrb + 1), 256, 0, s>>>(A, fl, j0, buf, P.wide_bstride);
    RQ_CUDA(cudaGetLastError());
    P.launches += nrb > 0 ? 2 : 1;
  }
}

template <class T>
void launch_factor_t(Problem& P, double cM, double cC, bool tc = false, bool indef = false,
                     double cMi = 0.0, double cCi = 0.0) {
  Plan& L = P.plan;
  cudaStream_t s = P.stream;
  FrontArgs<T> A = front_args<T>(P);
  A.indef = indef ? 1 : 0;
  constexpr bool cplx = std::is_same<T, zd>::value;
  const int32_t* piv_fronts = cplx ? P.cx.piv_fronts.p : P.piv_fronts.p;
  const std::vector<int32_t>& piv_lvl = cplx ? P.cx.piv_lvl : P.piv_lvl;
  const int4* rows = (const int4*)P.row_items.p;
  const int4* tiles = (const int4*)P.tile_items.p;
  for (int l = 0; l < L.nlevels; ++l) {
    int b = L.lvl_ptr[l], cnt = L.lvl_ptr[l + 1] - b;
    // several CTAs per front on levels with few fronts (about two CTAs per SM)
    const int nsplit = std::max(1, std::min(P.lvl_maxF[l] / 32, (2 * P.nsm + cnt - 1) / cnt));
    k_front_assemble<T><<<cnt * nsplit, 256, 0, s>>>(A, b, nsplit, P.rowptr_n.p, P.fpos.p, P.Kn.p,
                                                     P.Mn.p, P.Cn.p, cM, cC, cMi, cCi);
    RQ_CUDA(cudaGetLastError());
    const int nsm = piv_lvl[3 * l + 1] - piv_lvl[3 * l];
    const int nbig = piv_lvl[3 * l + 2] - piv_lvl[3 * l + 1];
    const int nwide = piv_lvl[3 * l + 3] - piv_lvl[3 * l + 2];
    if (nsm > 0) {
      k_pivot_factor<T><<<nsm, 256, sizeof(T) * (size_t)P.lvl_maxK[l], s>>>(
          A, piv_fronts + piv_lvl[3 * l]);
      RQ_CUDA(cudaGetLastError());
      ++P.launches;
    }
    if (nbig > 0) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)(nbig * kClusterCTAs));
      cfg.blockDim = dim3(256);
      cfg.dynamicSmemBytes =
          sizeof(T) * 32 * (size_t)std::min(P.lvl_maxK[l], cplx ? kClusterMaxKc : kClusterMaxK);
      cfg.stream = s;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = kClusterCTAs;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      const int32_t* fl = piv_fronts + piv_lvl[3 * l + 1];
      RQ_CUDA(cudaLaunchKernelEx(&cfg, k_pivot_cluster<T>, A, fl));
      ++P.launches;
    }
    if (nwide > 0) launch_wide_pivots<T>(P, A, piv_fronts + piv_lvl[3 * l + 2], nwide, l);
    ++P.launches;
    if (tc) {
      launch_tc_level(P, l);
      continue;
    }
    int rb = P.row_lvl[l], rc = P.row_lvl[l + 1] - rb;
    int tb = P.tile_lvl[l], tc = P.tile_lvl[l + 1] - tb;
    const int kl = std::max(1, P.lvl_maxK[l]);
    size_t smem = sizeof(T) * 16 * (size_t)kl;
    T* gout = nullptr;   // pivot blocks too wide for shared memory: a global buffer
    if (smem > kPanelSmemMax) {
      gout = reinterpret_cast<T*>(P.panel_scratch.p);
      smem = 0;
    }
    if (rc > 0) {
      k_panel_rows<T><<<rc, 256, smem, s>>>(A, rows, rb, 0, gout, kl);   // L21
      RQ_CUDA(cudaGetLastError());
      ++P.launches;
    }
    if (tc > 0) {
      k_schur_tile<T><<<tc, 256, 0, s>>>(A, tiles, tb);                 // U -= L21 D L21^T
      RQ_CUDA(cudaGetLastError());
      ++P.launches;
    }
    if (rc > 0) {
      k_panel_rows<T><<<rc, 256, smem, s>>>(A, rows, rb, 1, gout, kl);   // W = L21 inv(L11)
      RQ_CUDA(cudaGetLastError());
      ++P.launches;
    }
  }
}

void prepare_factor(Problem& P, int precision) {
  if (precision == RIGAQEP_FP64) return;
  Plan& L = P.plan;
  if (P.Lval32.n < (size_t)L.l_total) {   // FP32 factor storage on first use
    P.Lval32.alloc(L.l_total);
    P.Uval32.alloc(L.u_total);
    P.Dinv32.alloc(L.N);
    P.Dval32.alloc(L.N);
    P.yvec32.alloc(L.upd_idx.size());
    P.zbuf32.alloc(L.N);
    P.ir_y.alloc(L.N);
    P.ir_r32.alloc(L.N);
  }
  if (precision == RIGAQEP_TF32_IR || precision == RIGAQEP_BF16_IR)
    tc_plan(P, precision == RIGAQEP_BF16_IR);
}

void launch_factor(Problem& P, double sigma, int precision) {
  prepare_factor(P, precision);
  if (precision != RIGAQEP_FP64) {
    const bool tc = precision == RIGAQEP_TF32_IR || precision == RIGAQEP_BF16_IR;
    launch_factor_t<float>(P, sigma * sigma, sigma, tc);
    if (tc) tc_tuning_done(P);
  } else {
    launch_factor_t<double>(P, sigma * sigma, sigma);
  }
}

void launch_factor_gep(Problem& P, double mu) {
  launch_factor_t<double>(P, -mu, 0.0, false, true);
}

// Q(s) = K + s C + s^2 M at s = sr + i si, complex symmetric LDL^T (FP64)
void launch_factor_complex(Problem& P, double sr, double si) {
  Plan& L = P.plan;
  if (P.cx.Lval.n < (size_t)L.l_total) {   // complex factor storage on first use
    P.cx.Lval.alloc(L.l_total);
    P.cx.Uval.alloc(L.u_total);
    P.cx.Dinv.alloc(L.N);
    P.cx.Dval.alloc(L.N);
    P.cx.yvec.alloc(L.upd_idx.size());
    P.cx.zbuf.alloc(L.N);
    P.cx.y.alloc(L.N);
  }
  launch_factor_t<zd>(P, sr * sr - si * si, sr, false, false, 2.0 * sr * si, si);
}

void fb_plan(Problem& P) {
  Plan& L = P.plan;
  // per-front-position gather lists of the children's update entries
  std::vector<int32_t> gbase(L.nsuper + 1, 0);
  for (int s = 0; s < L.nsuper; ++s)
    gbase[s + 1] = gbase[s] + (L.sptr[s + 1] - L.sptr[s]) + (L.upd_ptr[s + 1] - L.upd_ptr[s]);
  std::vector<int32_t> cnt(gbase[L.nsuper] + 1, 0);
  for (int s = 0; s < L.nsuper; ++s)
    for (int ci = L.child_ptr[s]; ci < L.child_ptr[s + 1]; ++ci) {
      int c = L.child_idx[ci];
      for (int q = L.upd_ptr[c]; q < L.upd_ptr[c + 1]; ++q) ++cnt[gbase[s] + L.relmap[q] + 1];
    }
  std::vector<int32_t> gptr(cnt.size(), 0);
  for (size_t i = 1; i < cnt.size(); ++i) gptr[i] = gptr[i - 1] + cnt[i];
  std::vector<int32_t> gsrc(gptr.back()), fill(gptr.begin(), gptr.end() - 1);
  for (int s = 0; s < L.nsuper; ++s)
    for (int ci = L.child_ptr[s]; ci < L.child_ptr[s + 1]; ++ci) {   // child order
      int c = L.child_idx[ci];
      for (int q = L.upd_ptr[c]; q < L.upd_ptr[c + 1]; ++q) gsrc[fill[gbase[s] + L.relmap[q]]++] = q;
    }
  std::vector<int32_t> fwd, bwd;
  P.fwd_lvl.assign(L.nlevels + 1, 0);
  P.bwd_lvl.assign(L.nlevels + 1, 0);
  P.fwd_rc.assign(L.nlevels, 1);
  for (int l = 0; l < L.nlevels; ++l) {
    // 128-row forward items on levels whose pivot blocks are all small
    P.fwd_rc[l] = P.lvl_maxK[l] <= 64 ? 4 : 1;
    const int rows = 32 * P.fwd_rc[l];
    for (int q = L.lvl_ptr[l]; q < L.lvl_ptr[l + 1]; ++q) {
      int s = L.lvl_nodes[q];
      int a = L.sptr[s], k = L.sptr[s + 1] - a, u = L.upd_ptr[s + 1] - L.upd_ptr[s];
      int32_t lo = (int32_t)(uint32_t)(L.loff[s] & 0xffffffffll), hi = (int32_t)(L.loff[s] >> 32);
      int nkid = gptr[gbase[s + 1]] - gptr[gbase[s]];   // children's update entries
      for (int r = 0; r < k + u; r += rows)
        fwd.insert(fwd.end(), {s, r, std::min(rows, k + u - r), a, k, u, gbase[s], L.upd_ptr[s],
                               lo, hi, nkid, P.fwd_rc[l]});
      // backward items of 32 pivot columns; in the dependency-driven levels
      // the fronts of at least kBwdHalfRows rows take items of at most 16
      // (balanced), which the sweep runs with two lanes per column
      const int bw = l >= kDepLevel && k + u >= kBwdHalfRows ? (k + (k + 15) / 16 - 1) / ((k + 15) / 16)
                                                             : 32;
      for (int c = 0; c < k; c += bw)
        bwd.insert(bwd.end(), {s, c, std::min(bw, k - c), a, k, u, L.upd_ptr[s], 0, lo, hi, 0, 0});
    }
    P.fwd_lvl[l + 1] = (int32_t)(fwd.size() / 12);
    P.bwd_lvl[l + 1] = (int32_t)(bwd.size() / 12);
  }
  // blocks of the dependency-driven launches: as many as fit on the GPU at
  // once (more would only queue behind the resident ones)
  {
    int fa = 0, ba = 0;
    P.dep_maxK = 1;
    for (int l = kDepLevel; l < L.nlevels; ++l) P.dep_maxK = std::max(P.dep_maxK, P.lvl_maxK[l]);
    // the gathered right-hand side of the widest pivot block (above 48 KB on
    // the largest meshes)
    if (sizeof(double) * (size_t)P.dep_maxK > 48 * 1024)
      smem_at_least((const void*)k_fb_fwd_dep<double>, sizeof(double) * (size_t)P.dep_maxK);
    if (sizeof(float) * (size_t)P.dep_maxK > 48 * 1024)
      smem_at_least((const void*)k_fb_fwd_dep<float>, sizeof(float) * (size_t)P.dep_maxK);
    RQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &fa, k_fb_fwd_dep<double>, 256, sizeof(double) * (size_t)P.dep_maxK));
    RQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ba, k_fb_bwd_dep<double>, 256,
                                                          bwd_smem<double>(8)));
    P.dep_grid_fwd = std::max(1, fa) * P.nsm;
    P.dep_grid_bwd = std::max(1, ba) * P.nsm;
  }
  P.fwd_items.upload(fwd, P.stream);
  P.bwd_items.upload(bwd, P.stream);
  // dependency-driven sweeps of the levels from kDepLevel up: forward items
  // of the children inside that range, backward items per supernode, and
  // the backward items root level first (the order of their tickets)
  std::vector<int32_t> nf(L.nsuper, 0), nb(L.nsuper, 0), kid(L.nsuper, 0), border;
  for (size_t q = 0; q < fwd.size(); q += 12) ++nf[fwd[q]];
  for (size_t q = 0; q < bwd.size(); q += 12) ++nb[bwd[q]];
  for (int sn = 0; sn < L.nsuper; ++sn)
    if (L.level[sn] >= kDepLevel && L.parent[sn] >= 0) kid[L.parent[sn]] += nf[sn];
  for (int l = L.nlevels - 1; l >= kDepLevel; --l)
    for (int q = P.bwd_lvl[l]; q < P.bwd_lvl[l + 1]; ++q) border.push_back(q);
  P.fb_parent.upload(L.parent, P.stream);
  P.fb_kid_items.upload(kid, P.stream);
  P.fb_bwd_items.upload(nb, P.stream);
  P.fb_border.upload(border, P.stream);
  P.fb_counters.alloc(2 * (size_t)L.nsuper + 4);
  RQ_CUDA(cudaMemsetAsync(P.fb_counters.p, 0, sizeof(unsigned) * (2 * (size_t)L.nsuper + 4),
                          P.stream));
  P.fb_epoch = 0;
  P.fb_gptr.upload(gptr, P.stream);
  P.fb_gsrc.upload(gsrc, P.stream);
  P.zbuf.alloc(L.N);
  P.wbuf.alloc(1);
}

template <class T>
void launch_fb_t(Problem& P, T* xn, double sigma, const typename RealOf<T>::type* vu,
                 typename RealOf<T>::type* ru, typename RealOf<T>::type* rl, double uscale = 1.0,
                 double sigma_i = 0.0) {
  Plan& L = P.plan;
  cudaStream_t s = P.stream;
  FBArgs<T> A = fb_args<T>(P);
  constexpr bool cplx = std::is_same<T, zd>::value;
  // levels below ldep run one launch each (all levels for the complex factor)
  const int ldep = cplx ? L.nlevels : std::min(kDepLevel, L.nlevels);
  FBDep D{P.fb_parent.p, P.fb_kid_items.p, P.fb_bwd_items.p, P.fb_counters.p,
          P.fb_counters.p + L.nsuper, P.fb_counters.p + 2 * L.nsuper, ++P.fb_epoch, P.status.p};
  for (int l = 0; l < ldep; ++l) {
    int ib = P.fwd_lvl[l], ic = P.fwd_lvl[l + 1] - ib;
    const size_t sm = sizeof(T) * (size_t)P.lvl_maxK[l];
    if (P.fwd_rc[l] == 4)
      launch_pdl(k_fb_fwd<T, 4>, dim3(ic), dim3(256), sm, s, A, ib, (const T*)xn);
    else
      launch_pdl(k_fb_fwd<T, 1>, dim3(ic), dim3(256), sm, s, A, ib, (const T*)xn);
    ++P.launches;
  }
  if constexpr (!cplx) if (ldep < L.nlevels) {
    const int ib = P.fwd_lvl[ldep], ic = P.fwd_lvl[L.nlevels] - ib;
    const size_t sm = sizeof(T) * (size_t)P.dep_maxK;
    launch_pdl(k_fb_fwd_dep<T>, dim3((unsigned)std::min(ic, P.dep_grid_fwd)), dim3(256), sm, s, A,
               D, ib, ic, (const T*)xn);
    const int nb = (int)P.fb_border.n;
    D.ticket += 2;
    launch_pdl(k_fb_bwd_dep<T>, dim3((unsigned)std::min(nb, P.dep_grid_bwd)), dim3(256),
               bwd_smem<T>(8), s, A, D, (const int32_t*)P.fb_border.p, nb, xn, sigma, vu, ru, rl,
               uscale);
    P.launches += 2;
  }
  for (int l = ldep - 1; l >= 0; --l) {
    int ib = P.bwd_lvl[l], ic = P.bwd_lvl[l + 1] - ib;
    bool wide = ic < 2 * P.nsm;
    if constexpr (cplx) wide = true;   // eight warps per item (the complex blocks use more registers)
    if (wide) {
      launch_pdl(k_fb_bwd<T, 8>, dim3(ic), dim3(256), bwd_smem<T>(8), s, A, ib, xn, sigma, vu, ru,
                 rl, uscale, sigma_i);
    } else {
      if constexpr (!cplx)
        launch_pdl(k_fb_bwd<T, 4>, dim3(ic), dim3(128), bwd_smem<T>(4), s, A, ib, xn, sigma, vu,
                   ru, rl, uscale, sigma_i);
    }
    ++P.launches;
  }
}

// FP64 iterative refinement with the FP32 factors: x_0 = 0, r_0 = y;
//   d = Q32^{-1} r_i (FP32 sweeps),  x_{i+1} = x_i + d (FP64),
//   r_{i+1} = y - Q(s) x_{i+1} (FP64 residual from the assembled K, M, C),
// for a fixed number of steps chosen when the factor was made.
void launch_fb_ir(Problem& P, double* xn, double sigma, const double* vu, double* ru, double* rl,
                  double uscale) {
  Plan& L = P.plan;
  cudaStream_t s = P.stream;
  const int64_t N = L.N;
  const unsigned g = (unsigned)((N + 255) / 256);
  RQ_CUDA(cudaMemcpyAsync(P.ir_y.p, xn, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
  k_to_f32<<<g, 256, 0, s>>>(P.ir_y.p, P.ir_r32.p, N);
  RQ_CUDA(cudaGetLastError());
  P.launches += 1;
  for (int it = 0; it < P.n_ir; ++it) {
    launch_fb_t<float>(P, P.ir_r32.p, sigma, nullptr, nullptr, nullptr);
    k_ir_accum<<<g, 256, 0, s>>>(xn, P.ir_r32.p, N, it == 0 ? 1 : 0);
    RQ_CUDA(cudaGetLastError());
    P.launches += 1;
    if (it + 1 < P.n_ir) {
      k_ir_residual<<<(unsigned)((N * 8 + 255) / 256), 256, 0, s>>>(
          P.rowptr_n.p, P.col_n.p, P.Kn.p, P.Mn.p, P.Cn.p, sigma * sigma, sigma, xn, P.ir_y.p,
          P.ir_r32.p, N);
      RQ_CUDA(cudaGetLastError());
      P.launches += 1;
    }
  }
  if (ru) {
    k_op_out<<<g, 256, 0, s>>>(xn, sigma, vu, ru, rl, N, uscale);
    RQ_CUDA(cudaGetLastError());
    P.launches += 1;
  }
}

void launch_fb_complex(Problem& P, void* xn, double sr, double si, const double* vu, double* ru,
                       double* rl) {
  launch_fb_t<zd>(P, static_cast<zd*>(xn), sr, vu, ru, rl, 1.0, si);
}

void launch_fb(Problem& P, double* xn, double sigma, const double* vu, double* ru, double* rl,
               double uscale) {
  if (P.fact_fp32)
    launch_fb_ir(P, xn, sigma, vu, ru, rl, uscale);
  else
    launch_fb_t<double>(P, xn, sigma, vu, ru, rl, uscale);
}

// Relative residuals ||y - Q x_k|| / ||y|| of the refinement steps k = 1, 2,
// ... on a seeded right-hand side (host-side norms), until the residual
// reaches `target`, stops falling by half, or `max_steps` steps; used to
// choose the number of refinement steps after an FP32 factorisation.
std::vector<double> ir_history(Problem& P, double sigma, int max_steps, double target,
                               uint64_t seed) {
  Plan& L = P.plan;
  cudaStream_t s = P.stream;
  const int64_t N = L.N;
  DBuf<double> y, x, r;
  y.alloc(N);
  x.alloc(N);
  r.alloc(N);
  const unsigned g = (unsigned)((N + 255) / 256);
  const unsigned gr = (unsigned)((N * 8 + 255) / 256);
  k_probe_rhs<<<g, 256, 0, s>>>(seed, y.p, N);
  RQ_CUDA(cudaGetLastError());
  k_to_f32<<<g, 256, 0, s>>>(y.p, P.ir_r32.p, N);
  RQ_CUDA(cudaGetLastError());
  std::vector<double> hy(N), hr(N), hist;
  RQ_CUDA(cudaMemcpyAsync(hy.data(), y.p, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
  RQ_CUDA(cudaStreamSynchronize(s));
  double ny = 0.0;
  for (int64_t i = 0; i < N; ++i) ny += hy[i] * hy[i];
  ny = std::sqrt(ny);
  for (int k = 1; k <= max_steps; ++k) {
    launch_fb_t<float>(P, P.ir_r32.p, sigma, nullptr, nullptr, nullptr);
    k_ir_accum<<<g, 256, 0, s>>>(x.p, P.ir_r32.p, N, k == 1 ? 1 : 0);
    RQ_CUDA(cudaGetLastError());
    k_ir_residual64<<<gr, 256, 0, s>>>(P.rowptr_n.p, P.col_n.p, P.Kn.p, P.Mn.p, P.Cn.p,
                                        sigma * sigma, sigma, x.p, y.p, r.p, N);
    RQ_CUDA(cudaGetLastError());
    k_to_f32<<<g, 256, 0, s>>>(r.p, P.ir_r32.p, N);
    RQ_CUDA(cudaGetLastError());
    RQ_CUDA(cudaMemcpyAsync(hr.data(), r.p, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
    RQ_CUDA(cudaStreamSynchronize(s));
    double nr = 0.0;
    for (int64_t i = 0; i < N; ++i) nr += hr[i] * hr[i];
    hist.push_back(std::sqrt(nr) / ny);
    if (hist.back() <= target) break;
    if (k > 1 && !(hist.back() < 0.5 * hist[k - 2])) break;
  }
  return hist;
}

void launch_gather(const int32_t* idx, const double* src, double* dst, int64_t n, int32_t ld_in,
                   int32_t ncol, cudaStream_t s) {
  for (int c = 0; c < ncol; ++c) {
    k_gather<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(idx, src + (int64_t)c * ld_in,
                                                          dst + (int64_t)c * n, n);
    RQ_CUDA(cudaGetLastError());
  }
}

void launch_gather2(const int32_t* idx, const double* src, double* dst, int64_t n, cudaStream_t s) {
  k_gather2<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(idx, (const double2*)src, (double2*)dst, n);
  RQ_CUDA(cudaGetLastError());
}

void launch_scatter2(const int32_t* idx, const double* src, double* dst, int64_t n, cudaStream_t s) {
  k_scatter2<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(idx, (const double2*)src, (double2*)dst, n);
  RQ_CUDA(cudaGetLastError());
}

void launch_scatter(const int32_t* idx, const double* src, double* dst, int64_t n, cudaStream_t s) {
  k_scatter<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(idx, src, dst, n);
  RQ_CUDA(cudaGetLastError());
}

}  // namespace rq
