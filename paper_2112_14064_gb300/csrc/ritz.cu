// Rayleigh-Ritz step and Krylov-Schur truncation on the device (FP64).
//
// Input: the (m+1) x m projected matrix of a Krylov decomposition
//   S V_m = V_m H_m + h_{m+1,m} v_{m+1} e_m^T   (paper Eq. Arnoldi; after a
//   restart the leading k x k block is quasi-triangular with a spike row).
// Ritz values theta of H_m approximate the eigenvalues of the shift-and-invert
// operator (Eq. ArnoldiRitz); lambda = s + 1/theta (Section 4.1.1).  The
// restart keeps the invariant subspace of the wanted Ritz values (Krylov-Schur,
// Section 4.1.3, which the paper cites without details).
//
// A cluster of three CTAs of four warps each (one warp per SM sub-partition,
// so the FP64 row and column updates use all four FP64 pipes of an SM).  The
// first CTA does the whole step in its shared memory:
//   1. Householder reduction of H_m to Hessenberg form, Z accumulated;
//   2. Francis double-shift QR to real Schur form T = Z^T H_m Z, 2x2 blocks
//      standardised (equal diagonal for complex pairs, split when real);
//   3. rank of every Ritz value by |lambda - s| (Im > 0 first on ties);
//   4. eigenvectors of the wanted values by back-substitution on T, Ritz
//      estimates |h_{m+1,m} e_m^T Z y| / (|theta| ||y||);
//   5. restart: the wanted blocks are moved to the top of T by adjacent block
//      swaps (each swap solves the small Sylvester equation A X - X B = C and
//      applies the orthogonal factor of [X; -I]); the new projected matrix is
//      [T_kk ; h_{m+1,m} Z(m,1:k)] and the kept basis is V Z(:,1:k);
//   6. locking: converged kept blocks move to the front and their entries of
//      the spike row are set to zero, so the projected matrix stays block
//      upper triangular and later steps reduce and iterate only on the
//      trailing active block (the locked Schur part is left as it is).
// During step 2 the other two CTAs apply, one sweep behind, the updates that
// lie outside the active window: the second CTA accumulates Z in its own
// shared memory, the third updates the rows above and the columns right of
// the window in the first CTA's T through distributed shared memory.  The
// first CTA hands each sweep over in a double-buffered batch (its reflectors
// and the rotations of the 2 x 2 blocks deflated before it) and goes on with
// the next sweep.
#include <cooperative_groups.h>

#include "internal.h"
#include "nr_math.cuh"
#include "tma.cuh"

namespace rq {
namespace {

constexpr double kEps = 2.220446049250313e-16;
constexpr int NT = 128;   // threads of each Ritz CTA
constexpr int kRitzCTAs = 3;   // cluster: the Ritz CTA, the Z CTA and the off-window T CTA
constexpr int kMaxRot = 48;    // rotations per batch (2 x 2 deflations between sweeps)

struct RitzArgs {
  const double* H;   // (m+1) x m, column-major, ld = m+1
  double* Hnew;      // restart matrix, same layout
  double* Q;         // m x k kept Schur vectors, ld = m
  double* Y;         // when finishing: m x neig eigenvectors of H_m (re, im interleaved)
  RitzOut* out;
  int m, neig, kwant, final_pass, lock;   // final_pass: 0 restart, 1 finish, 2 finish if converged
  double sigma, tol;
  uint32_t wait_limit;   // polls of a batch barrier before giving up
  double tscale;         // lambda = sigma + tscale / theta (scaled pencil: the scaling factor)
};

struct Smem {
  double* T;   // m x m, column-major, leading dimension ld
  double* Z;   // m x m, leading dimension ld
  int ld;      // m rounded up to odd: row-wise lane access hits distinct banks
  double* v;   // Householder vector (m)
  double* wr;  // Ritz values (Schur order)
  double* wi;
  int* rank;
  int* sel;
  int* cflag;  // converged flag of each Schur position
  double* red; // 4 partial sums
  char* batch; // two batches of deferred QR work (BatchHdr, Rot[kMaxRot], Refl[])
};

#define TT(r, c) S.T[(r) + S.ld * (c)]
#define ZZ(r, c) S.Z[(r) + S.ld * (c)]

// Householder reflector for x[0..n): (I - tau v v^T) x = beta e_0, v[0] = 1.
// All threads compute it redundantly from the same data.
__device__ void house(const double* x, int n, double* v, double& tau, double& beta) {
  double alpha = x[0], sg = 0.0;
  for (int i = 1; i < n; ++i) sg += x[i] * x[i];
  v[0] = 1.0;
  if (sg == 0.0) {
    tau = 0.0;
    beta = alpha;
    for (int i = 1; i < n; ++i) v[i] = 0.0;
    return;
  }
  double nr = sqrt_nr(alpha * alpha + sg);
  beta = alpha <= 0.0 ? nr : -nr;
  double d = alpha - beta;
  double rd = rcp_nr(d);
  for (int i = 1; i < n; ++i) v[i] = x[i] * rd;
  tau = div_nr(beta - alpha, beta);
}

// T columns c0..c0+n-1 (rows r0..r1-1) and Z columns c0..c0+n-1 (all m rows)
// <- cols P in one pass, one row per thread: keeps all four warps busy.
__device__ void apply_right_tz(double* T, double* Z, int m, int ld, const double* v, double tau,
                               int n, int c0, int r0, int r1, int lane) {
  if (tau == 0.0) return;
  int nt = r1 - r0;
  for (int q = lane; q < nt + m; q += NT) {
    double* A = q < nt ? T : Z;
    int r = q < nt ? r0 + q : q - nt;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += v[i] * A[r + ld * (c0 + i)];
    s *= tau;
    for (int i = 0; i < n; ++i) A[r + ld * (c0 + i)] -= s * v[i];
  }
}

// rows r0..r0+n-1 of A (leading dimension ld) <- P rows, columns c0..c1-1,
// threads over columns
__device__ void apply_left(double* A, int ld, const double* v, double tau, int n, int r0, int c0,
                           int c1, int lane) {
  if (tau == 0.0) return;
  for (int c = c0 + lane; c < c1; c += NT) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += v[i] * A[(r0 + i) + ld * c];
    s *= tau;
    for (int i = 0; i < n; ++i) A[(r0 + i) + ld * c] -= s * v[i];
  }
}

// Deferred QR work handed from the Ritz CTA to the helper CTAs, one batch per
// sweep: the rotations of the 2 x 2 blocks standardised since the last sweep
// (applied first, in order), then the sweep's reflectors in (round, bulge)
// order.
struct Refl;
struct BatchHdr {
  int nrot;          // rotations
  int sweep;         // 1: reflectors of a sweep on the window [l, hi] follow
  int l, hi, nb, rounds;
  int end;           // last batch of the QR iteration
  int pad;
};
struct Rot {         // G = [[c, -s], [s, c]] on rows/columns j, j+1
  double c, s;
  int j, pad;
};
constexpr size_t kReflOff = (sizeof(BatchHdr) + kMaxRot * sizeof(Rot) + 15) / 16 * 16;

// The Ritz CTA's side of the batch queue.  Two batch buffers live in its
// shared memory; `full` barriers (one arrival) in each helper CTA, `empty`
// barriers (one arrival per helper) and `done` in the Ritz CTA.  Every thread
// keeps the same copy of the counters.
struct Queue {
  char* buf;         // batch 0; batch 1 follows at bbytes
  size_t bbytes;
  uint64_t* bars;    // [0..1] full, [2..3] empty, [4] done (same offsets in every CTA)
  int* err;          // shared flag: a bounded wait ran out
  uint32_t limit;    // polls of a barrier before a wait gives up
  int bq;            // batch being filled
  int nrot;          // its rotations so far
  bool open;         // its buffer has been released by the helpers
  __device__ BatchHdr* hdr(int b) const { return (BatchHdr*)(buf + (size_t)(b & 1) * bbytes); }
  __device__ Rot* rot(int b) const { return (Rot*)(buf + (size_t)(b & 1) * bbytes + sizeof(BatchHdr)); }
  __device__ Refl* refl(int b) const { return (Refl*)(buf + (size_t)(b & 1) * bbytes + kReflOff); }
};

// Makes the buffer of batch bq writable: its previous batch (bq - 2) has been
// copied by both helpers.
__device__ void q_acquire(Queue& Q, int lane) {
  if (Q.open) return;
  if (Q.bq >= 2 && lane == 0 &&
      !mbar_wait_cluster(&Q.bars[2 + (Q.bq & 1)], (uint32_t)(((Q.bq >> 1) - 1) & 1), Q.limit))
    *Q.err = 1;
  __syncthreads();
  Q.open = true;
  Q.nrot = 0;
}

// Completes batch bq (every thread's writes to it are done) and signals both
// helpers.
__device__ void q_publish(Queue& Q, int lane, int sweep, int l, int hi, int nb, int rounds, int end) {
  __syncthreads();
  if (lane == 0) {
    BatchHdr* h = Q.hdr(Q.bq);
    h->nrot = Q.nrot;
    h->sweep = sweep;
    h->l = l;
    h->hi = hi;
    h->nb = nb;
    h->rounds = rounds;
    h->end = end;
    h->pad = 0;
    fence_acq_rel_cluster();
    for (int r = 1; r < kRitzCTAs; ++r) mbar_arrive_remote(&Q.bars[Q.bq & 1], (uint32_t)r);
  }
  ++Q.bq;
  Q.open = false;
}

// G applied to the 2 x 2 block at j alone (T_jj..T_j+1,j+1 <- G^T T G); the
// rows right of it, the columns above it and Z are left to the helpers.
__device__ void rotate_block(Smem& S, int m, int j, double c, double s, int lane) {
  __syncthreads();
  if (lane == 0) {
    for (int col = j; col <= j + 1; ++col) {
      double a = TT(j, col), b = TT(j + 1, col);
      TT(j, col) = c * a + s * b;
      TT(j + 1, col) = -s * a + c * b;
    }
    for (int r = j; r <= j + 1; ++r) {
      double a = TT(r, j), b = TT(r, j + 1);
      TT(r, j) = c * a + s * b;
      TT(r, j + 1) = -s * a + c * b;
    }
  }
  __syncthreads();
}

// Plane rotation G = [[c, -s], [s, c]] on rows/cols j, j+1: T <- G^T T G, Z <- Z G
__device__ void rotate(Smem& S, int m, int j, double c, double s, int lane) {
  __syncthreads();
  for (int col = j + lane; col < m; col += NT) {
    double a = TT(j, col), b = TT(j + 1, col);
    TT(j, col) = c * a + s * b;
    TT(j + 1, col) = -s * a + c * b;
  }
  __syncthreads();
  for (int r = lane; r < m; r += NT) {
    if (r <= j + 1) {
      double a = TT(r, j), b = TT(r, j + 1);
      TT(r, j) = c * a + s * b;
      TT(r, j + 1) = -s * a + c * b;
    }
    double a = ZZ(r, j), b = ZZ(r, j + 1);
    ZZ(r, j) = c * a + s * b;
    ZZ(r, j + 1) = -s * a + c * b;
  }
  __syncthreads();
}

// Standardise the 2x2 diagonal block at j: split it (exact zero below the
// diagonal) when its eigenvalues are real, else make its diagonal equal.
// Returns true when the block stays a complex pair.  With a queue (during the
// QR iteration) only the block itself is rotated here and the rotation is
// appended to the open batch for the rest of T and for Z.
// Rotation (c, s) that standardises the 2x2 block at j (no synchronisation;
// any number of threads may compute it).  Returns 0 when the block is
// already split (T[j+1, j] = 0), 1 when its eigenvalues are real, 2 when they
// are a complex pair.
__device__ int std2_params(const Smem& S, int j, double& c, double& s) {
  double a = TT(j, j), b = TT(j, j + 1), e = TT(j + 1, j), d = TT(j + 1, j + 1);
  if (e == 0.0) return 0;
  double hp = 0.5 * (a - d);
  double disc = hp * hp + b * e;
  bool cplx;
  if (disc >= 0.0) {
    // eigenvector of the eigenvalue l1; g1 = (c, s) spans it
    double rt = sqrt_nr(disc);
    double l1 = 0.5 * (a + d) + (hp >= 0.0 ? rt : -rt);
    double x1 = b, y1 = l1 - a;      // from the first row
    double x2 = l1 - d, y2 = e;      // from the second row
    double n1 = x1 * x1 + y1 * y1, n2 = x2 * x2 + y2 * y2;
    double x = n1 >= n2 ? x1 : x2, y = n1 >= n2 ? y1 : y2;
    double rn = rcp_nr(sqrt_nr(x * x + y * y));
    c = x * rn;
    s = y * rn;
    cplx = false;
  } else {
    // T'11 - T'22 = cos(2t)(a - d) + sin(2t)(b + e) = 0: with
    // (cos 2t, sin 2t) = (q, p)/r, half-angle formulas give (cos t, sin t)
    double pp = -(a - d), qq = b + e;
    double r2 = pp * pp + qq * qq;
    if (r2 == 0.0) {
      c = 1.0;
      s = 0.0;
    } else {
      double rr = rcp_nr(sqrt_nr(r2));
      double c2 = qq * rr, s2 = pp * rr;
      if (c2 >= 0.0) {
        c = sqrt_nr(0.5 * (1.0 + c2));
        s = s2 * 0.5 * rcp_nr(c);
      } else {
        s = sqrt_nr(0.5 * (1.0 - c2));
        if (s2 < 0.0) s = -s;
        c = s2 * 0.5 * rcp_nr(s);
      }
    }
    cplx = true;
  }
  return cplx ? 2 : 1;
}

__device__ bool standardize2(Smem& S, int m, int j, int lane, Queue* q = nullptr) {
  double c, s;
  const int kind = std2_params(S, j, c, s);
  if (kind == 0) return false;
  const bool cplx = kind == 2;
  if (q) {
    rotate_block(S, m, j, c, s, lane);
    if (lane == 0) {
      Rot* rt = q->rot(q->bq) + q->nrot;
      rt->c = c;
      rt->s = s;
      rt->j = j;
      rt->pad = 0;
    }
    ++q->nrot;
  } else {
    rotate(S, m, j, c, s, lane);
  }
  if (!cplx) {
    if (lane == 0) TT(j + 1, j) = 0.0;
  } else if (lane == 0) {
    double avg = 0.5 * (TT(j, j) + TT(j + 1, j + 1));
    TT(j, j) = avg;
    TT(j + 1, j + 1) = avg;
  }
  __syncthreads();
  return cplx;
}

// Reflectors of the swap of the adjacent diagonal blocks at j (size n1) and
// j+n1 (size n2): the Sylvester equation A X - X B = C, then the Householder
// QR of [X; -I] (n2 reflectors of length n - q in vh[q], tau[q]).  No
// synchronisation; any number of threads may compute it.
__device__ void swap_setup(const Smem& S, int j, int n1, int n2, double tnorm, double (&vh)[2][4],
                           double (&tau)[2]) {
  int n = n1 + n2;
  double A[2][2], B[2][2], Cm[2][2];
  for (int r = 0; r < n1; ++r)
    for (int c = 0; c < n1; ++c) A[r][c] = TT(j + r, j + c);
  for (int r = 0; r < n2; ++r)
    for (int c = 0; c < n2; ++c) B[r][c] = TT(j + n1 + r, j + n1 + c);
  for (int r = 0; r < n1; ++r)
    for (int c = 0; c < n2; ++c) Cm[r][c] = TT(j + r, j + n1 + c);
  // Sylvester A X - X B = C, unknown X[r][c] at index r + n1*c
  int ns = n1 * n2;
  double G[4][5];
  for (int r = 0; r < n1; ++r)
    for (int c = 0; c < n2; ++c) {
      int row = r + n1 * c;
      for (int r2 = 0; r2 < n1; ++r2)
        for (int c2 = 0; c2 < n2; ++c2) {
          int cc = r2 + n1 * c2;
          double v = 0.0;
          if (c == c2) v += A[r][r2];
          if (r == r2) v -= B[c2][c];
          G[row][cc] = v;
        }
      G[row][ns] = Cm[r][c];
    }
  double smin = fmax(kEps * tnorm, 1e-300);
  for (int col = 0; col < ns; ++col) {
    int piv = col;
    for (int r = col + 1; r < ns; ++r)
      if (fabs(G[r][col]) > fabs(G[piv][col])) piv = r;
    if (piv != col)
      for (int c = 0; c <= ns; ++c) {
        double t = G[col][c];
        G[col][c] = G[piv][c];
        G[piv][c] = t;
      }
    if (fabs(G[col][col]) < smin) G[col][col] = G[col][col] >= 0.0 ? smin : -smin;
    double rp = rcp_nr(G[col][col]);
    for (int r = col + 1; r < ns; ++r) {
      double f = G[r][col] * rp;
      for (int c = col; c <= ns; ++c) G[r][c] -= f * G[col][c];
    }
  }
  double xs[4];
  for (int r = ns - 1; r >= 0; --r) {
    double t = G[r][ns];
    for (int c = r + 1; c < ns; ++c) t -= G[r][c] * xs[c];
    xs[r] = t * rcp_nr(G[r][r]);
  }
  // W = [X; -I] (n x n2); Householder QR, reflectors kept in vh
  double W[4][2];
  for (int r = 0; r < n1; ++r)
    for (int c = 0; c < n2; ++c) W[r][c] = xs[r + n1 * c];
  for (int r = 0; r < n2; ++r)
    for (int c = 0; c < n2; ++c) W[n1 + r][c] = (r == c) ? -1.0 : 0.0;
  for (int q = 0; q < n2; ++q) {
    double x[4];
    for (int i = q; i < n; ++i) x[i - q] = W[i][q];
    double beta;
    for (int i = 0; i < 4; ++i) vh[q][i] = 0.0;
    house(x, n - q, vh[q] + q, tau[q], beta);
    // apply to the remaining columns of W
    for (int c = q + 1; c < n2; ++c) {
      double s = 0.0;
      for (int i = q; i < n; ++i) s += vh[q][i] * W[i][c];
      s *= tau[q];
      for (int i = q; i < n; ++i) W[i][c] -= s * vh[q][i];
    }
  }
}

// Swap the adjacent diagonal blocks at j (size n1) and j+n1 (size n2).
__device__ void swap_blocks(Smem& S, int m, int j, int n1, int n2, double tnorm, int lane) {
  const int n = n1 + n2;
  double vh[2][4], tau[2];
  swap_setup(S, j, n1, n2, tnorm, vh, tau);
  __syncthreads();
  for (int q = 0; q < n2; ++q) {
    apply_left(S.T, S.ld, vh[q], tau[q], n, j, j, m, lane);
    __syncthreads();
    apply_right_tz(S.T, S.Z, m, S.ld, vh[q], tau[q], n, j, 0, j + n, lane);
    __syncthreads();
  }
  if (lane == 0)
    for (int r = j + n2; r < j + n; ++r)
      for (int c = j; c < j + n2; ++c) TT(r, c) = 0.0;
  __syncthreads();
  if (n2 == 2) standardize2(S, m, j, lane);
  if (n1 == 2) standardize2(S, m, j + n2, lane);
}

// ---- block reordering in parallel rounds ----
// In each round every unselected block directly above a selected block swaps
// with it; such pairs occupy disjoint diagonal ranges, so up to one pair per
// warp is swapped at once.  Each warp forms its pair's reflectors and
// standardising rotations; the updates then run in phases separated by CTA
// barriers: every warp's left (row) updates, then every warp's right (column)
// updates of T and Z.  Left updates of different pairs touch disjoint rows,
// right updates disjoint columns, and a left and a right update commute, so
// the result is that of the same swaps one after another.
constexpr int kMaxPairs = kMaxKrylov / 2;

// rows r0..r0+n-1 of A <- P rows, columns c0..c1-1, the lanes of one warp
__device__ void warp_apply_left(double* A, int ld, const double* v, double tau, int n, int r0,
                                int c0, int c1, int wl) {
  if (tau == 0.0) return;
  for (int c = c0 + wl; c < c1; c += 32) {
    double sd = 0.0;
    for (int i = 0; i < n; ++i) sd += v[i] * A[(r0 + i) + ld * c];
    sd *= tau;
    for (int i = 0; i < n; ++i) A[(r0 + i) + ld * c] -= sd * v[i];
  }
}

// T columns c0..c0+n-1 (rows 0..r1-1) and Z columns c0..c0+n-1 (all rows)
// <- cols P, the lanes of one warp
__device__ void warp_apply_right_tz(double* T, double* Z, int m, int ld, const double* v,
                                    double tau, int n, int c0, int r1, int wl) {
  if (tau == 0.0) return;
  for (int q = wl; q < r1 + m; q += 32) {
    double* A = q < r1 ? T : Z;
    int r = q < r1 ? q : q - r1;
    double sd = 0.0;
    for (int i = 0; i < n; ++i) sd += v[i] * A[r + ld * (c0 + i)];
    sd *= tau;
    for (int i = 0; i < n; ++i) A[r + ld * (c0 + i)] -= sd * v[i];
  }
}

// Moves the selected blocks (S.sel) to the top of T; returns their size.
__device__ int reorder_parallel(Smem& S, int m, double tnorm, int lane) {
  __shared__ int npair, pj[kMaxPairs], pn1[kMaxPairs], pn2[kMaxPairs];
  const int warp = lane >> 5, wl = lane & 31;
  constexpr int kW = NT / 32;
  for (int round = 0; round < 2 * m; ++round) {
    if (lane == 0) {
      // (unselected, selected) neighbours, top down, each block in one pair
      int np = 0, pos = 0, up = -1, un = 0;
      while (pos < m) {
        const int bs = (pos + 1 < m && TT(pos + 1, pos) != 0.0) ? 2 : 1;
        if (S.sel[pos] && up >= 0 && np < kMaxPairs) {
          pj[np] = up;
          pn1[np] = un;
          pn2[np] = bs;
          ++np;
          up = -1;
        } else {
          up = S.sel[pos] ? -1 : pos;
          un = bs;
        }
        pos += bs;
      }
      npair = np;
    }
    __syncthreads();
    const int np = npair;
    if (np == 0) break;
    for (int g0 = 0; g0 < np; g0 += kW) {
      const bool act = warp < np - g0;
      const int pi = g0 + warp;
      int j = 0, n1 = 0, n2 = 0, cf_sel[2] = {0, 0}, cf_oth[2] = {0, 0};
      double vh[2][4], tau[2] = {0.0, 0.0};
      if (act) {
        j = pj[pi];
        n1 = pn1[pi];
        n2 = pn2[pi];
        cf_oth[0] = S.cflag[j];
        cf_oth[1] = n1 == 2 ? S.cflag[j + 1] : 0;
        cf_sel[0] = S.cflag[j + n1];
        cf_sel[1] = n2 == 2 ? S.cflag[j + n1 + 1] : 0;
        swap_setup(S, j, n1, n2, tnorm, vh, tau);
      }
      const int n = n1 + n2;
      __syncthreads();
      for (int q = 0; q < 2; ++q) {
        if (act && q < n2) warp_apply_left(S.T, S.ld, vh[q], tau[q], n, j, j, m, wl);
        __syncthreads();
        if (act && q < n2) warp_apply_right_tz(S.T, S.Z, m, S.ld, vh[q], tau[q], n, j, j + n, wl);
        __syncthreads();
      }
      if (act && wl == 0)
        for (int r = j + n2; r < j + n; ++r)
          for (int c = j; c < j + n2; ++c) TT(r, c) = 0.0;
      __syncthreads();
      // standardise the new blocks at j (size n2) and j + n2 (size n1)
      int rk[2] = {0, 0}, rj[2] = {j, j + n2};
      double rc[2] = {1.0, 1.0}, rs[2] = {0.0, 0.0};
      if (act) {
        if (n2 == 2) rk[0] = std2_params(S, j, rc[0], rs[0]);
        if (n1 == 2) rk[1] = std2_params(S, j + n2, rc[1], rs[1]);
      }
      __syncthreads();
      for (int b = 0; b < 2; ++b)   // left: rows j', j'+1, columns from j'
        if (act && rk[b])
          for (int col = rj[b] + wl; col < m; col += 32) {
            const double x = TT(rj[b], col), y = TT(rj[b] + 1, col);
            TT(rj[b], col) = rc[b] * x + rs[b] * y;
            TT(rj[b] + 1, col) = -rs[b] * x + rc[b] * y;
          }
      __syncthreads();
      for (int b = 0; b < 2; ++b)   // right: columns j', j'+1 of T (rows <= j'+1) and Z
        if (act && rk[b])
          for (int r = wl; r < m; r += 32) {
            if (r <= rj[b] + 1) {
              const double x = TT(r, rj[b]), y = TT(r, rj[b] + 1);
              TT(r, rj[b]) = rc[b] * x + rs[b] * y;
              TT(r, rj[b] + 1) = -rs[b] * x + rc[b] * y;
            }
            const double x = ZZ(r, rj[b]), y = ZZ(r, rj[b] + 1);
            ZZ(r, rj[b]) = rc[b] * x + rs[b] * y;
            ZZ(r, rj[b] + 1) = -rs[b] * x + rc[b] * y;
          }
      __syncthreads();
      if (act && wl == 0) {
        for (int b = 0; b < 2; ++b) {
          const int jj = rj[b];
          if (rk[b] == 1) {
            TT(jj + 1, jj) = 0.0;
          } else if (rk[b] == 2) {
            const double avg = 0.5 * (TT(jj, jj) + TT(jj + 1, jj + 1));
            TT(jj, jj) = avg;
            TT(jj + 1, jj + 1) = avg;
          }
        }
        // the selected block now starts at j; keep the flags in step
        for (int i = 0; i < n2; ++i) { S.sel[j + i] = 1; S.cflag[j + i] = cf_sel[i]; }
        for (int i = 0; i < n1; ++i) { S.sel[j + n2 + i] = 0; S.cflag[j + n2 + i] = cf_oth[i]; }
      }
      __syncthreads();
    }
  }
  int k = 0;
  while (k < m && S.sel[k]) ++k;
  return k;
}

// Sum over the CTA; every thread gets the result.
__device__ double block_sum(double v, double* red, int lane) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((lane & 31) == 0) red[lane >> 5] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int w = 0; w < NT / 32; ++w) s += red[w];
  __syncthreads();
  return s;
}

__device__ double frob(Smem& S, int m, int lane) {
  double s = 0.0;
  for (int i = lane; i < S.ld * m; i += NT) s += S.T[i] * S.T[i];   // padding rows are 0
  return sqrt(block_sum(s, S.red, lane));
}

// Reflector P = I - tau u u^T with P x = beta e_0 for x of length n (2 or 3):
// u = x - beta e_0, beta = -sign(x_0) ||x||, and u^T u = 2 beta (beta - x_0),
// so tau = 2 / u^T u = 1 / (beta (beta - x_0)): one square root, one reciprocal.
struct alignas(16) Refl {
  double u0, u1, u2, tau;
  int pos, n;
};

// The tests and the sign choice are integer operations on the bits (an FP64
// compare would cost a 64-cycle FP64 instruction on the round's critical
// chain).  n = 0 marks the identity (x_1 = x_2 = 0).
__device__ __forceinline__ void make_refl(double x0, double x1, double x2, int n, Refl& r) {
  if (n == 2) x2 = 0.0;
  const double q = fma(x0, x0, fma(x2, x2, x1 * x1));
  const long long b1 = __double_as_longlong(x1) << 1, b2 = __double_as_longlong(x2) << 1;
  if ((b1 | b2) == 0 || (__double_as_longlong(q) << 1) == 0) {
    r.u0 = 1.0; r.u1 = 0.0; r.u2 = 0.0; r.tau = 0.0; r.n = 0;
    return;
  }
  r.n = n;
  const double nr = sqrt_nr(q);
  // beta = -sign(x0) ||x|| (beta = ||x|| for x0 = +-0)
  const long long flip = __double_as_longlong(x0) > 0 ? (long long)0x8000000000000000ULL : 0LL;
  const double beta = __longlong_as_double(__double_as_longlong(nr) ^ flip);
  r.u0 = x0 - beta;
  r.u1 = x1;
  r.u2 = x2;
  r.tau = rcp_nr(-beta * r.u0);   // 1 / (beta (beta - x0))
}

// rows pos..pos+n-1 of column c of A (leading dimension ld) <- P (rows)
__device__ __forceinline__ void refl_col(double* A, int ld, const Refl& r, int c) {
  double* a = A + r.pos + ld * c;
  double s = r.u0 * a[0] + r.u1 * a[1];
  if (r.n == 3) s += r.u2 * a[2];
  s *= r.tau;
  a[0] -= s * r.u0;
  a[1] -= s * r.u1;
  if (r.n == 3) a[2] -= s * r.u2;
}

// columns pos..pos+n-1 of row i of A <- (cols) P
__device__ __forceinline__ void refl_row(double* A, int ld, const Refl& r, int i) {
  double* a = A + i + ld * r.pos;
  double s = r.u0 * a[0] + r.u1 * a[ld];
  if (r.n == 3) s += r.u2 * a[2 * ld];
  s *= r.tau;
  a[0] -= s * r.u0;
  a[ld] -= s * r.u1;
  if (r.n == 3) a[2 * ld] -= s * r.u2;
}

// Real Schur form of the Hessenberg T by Francis double-shift sweeps.
//
// A sweep on the active window [l, hi] chases a chain of up to kBulges
// double-shift bulges (one per warp), each kBulgeGap rows behind the one
// ahead of it; with at most one bulge the sweep is the classical one.
// The bulges use the Francis shift pair of the trailing 2 x 2 block (bulge 0
// with the usual exceptional shift every 11th sweep).  Each round every bulge
// moves one position:
//   warp b: build its reflector and apply it from the right (columns
//           kq..kq+2, window rows up to kq+3);
//   barrier;
//   warp b: apply it from the left (rows kq..kq+2, window columns from kq-1);
//   barrier.
// With the bulges at least four rows apart the right-hand updates of one
// round touch disjoint columns and the left-hand updates disjoint rows; the
// only overlap between bulges (the rows of a bulge behind against the
// columns of the bulge ahead) sees the ahead bulge's right-hand update before
// the behind bulge's left-hand update, as in the one-bulge-at-a-time order.
// A left and a right application of one reflector commute.
//
// Only window entries are updated here.  The sweep's reflectors go to the
// helper CTAs, which apply them, in (round, bulge) order, to the columns
// right of the window, the rows above it and Z while this CTA runs the next
// sweep.  That is safe because an entry outside the window of one sweep is
// outside the window of every later sweep (later windows lie inside it or
// wholly above it), and the deflation tests read only diagonal and
// subdiagonal entries, which the helpers never write.
// Returns 0 when converged, 1 when the sweep limit was reached, 2 when a
// bounded wait on the helpers ran out.
constexpr int kBulges = NT / 32;
constexpr int kVecWarps = NT / 32 < 4 ? NT / 32 : 4;   // warps computing eigenvectors
constexpr int kBulgeGap = 4;

__host__ __device__ inline size_t batch_bytes(int m) {
  return kReflOff + sizeof(Refl) * (size_t)kBulges * (size_t)(m + 4 * kBulges);
}

// The deflation point of the active window [lock, hi]: the largest
// l in (lock, hi] whose subdiagonal entry is negligible against its two
// diagonal neighbours (|T(l, l-1)| <= eps (|T(l-1, l-1)| + |T(l, l)|)), or
// lock if there is none.  One subdiagonal entry per thread and a block
// maximum: each test is four FP64 instructions, which a scan down the
// window would chain once per row.  Returns the same value to every thread.
__device__ int deflation_point(const Smem& S, int lock, int hi, double tn, int lane) {
  __shared__ int wmax[NT / 32];
  int best = lock;
  for (int i = lock + 1 + lane; i <= hi; i += NT) {
    double sc = fabs(TT(i - 1, i - 1)) + fabs(TT(i, i));
    if (sc == 0.0) sc = tn;
    if (fabs(TT(i, i - 1)) <= kEps * sc) best = i;   // i increases: the last hit is the largest
  }
  best = __reduce_max_sync(0xffffffffu, best);
  if ((lane & 31) == 0) wmax[lane >> 5] = best;
  __syncthreads();
  int l = wmax[0];
#pragma unroll
  for (int w = 1; w < NT / 32; ++w) l = max(l, wmax[w]);
  __syncthreads();
  return l;
}

__device__ int francis(Smem& S, int m, int lane, int& sweeps, int lock, Queue& Q) {
  double tn = frob(S, m, lane);
  if (tn == 0.0) tn = 1.0;
  int hi = m - 1, its = 0, total = 0, status = 0;
  const int warp = lane >> 5, wl = lane & 31;
  while (hi >= lock) {
    const int l = hi > lock ? deflation_point(S, lock, hi, tn, lane) : lock;
    if (l > lock && lane == 0) TT(l, l - 1) = 0.0;
    __syncthreads();
    if (l == hi) { --hi; its = 0; continue; }
    if (l == hi - 1) {
      if (Q.open && Q.nrot == kMaxRot) q_publish(Q, lane, 0, 0, 0, 0, 0, 0);
      q_acquire(Q, lane);
      if (*Q.err) { status = 2; break; }
      standardize2(S, m, hi - 1, lane, &Q);
      hi -= 2;
      its = 0;
      continue;
    }
    if (++total > 40 * m) { status = 1; break; }
    ++its;
    const int nw = hi - l + 1;
    const int nb = max(1, min(kBulges, nw / (kBulgeGap + 2)));
    // this warp's shift pair (sum sh, product th): every bulge takes the
    // eigenvalues of the trailing 2 x 2 block (measured: fewer sweeps and
    // less time than shifts from the 2 x 2 blocks above it); bulge 0 takes
    // the exceptional shift every 11th sweep
    double sh = 0.0, th = 0.0;
    if (warp < nb) {
      int p = hi - 1;
      if (warp == 0 && its % 11 == 10) {
        double w = fabs(TT(hi, hi - 1)) + fabs(TT(hi - 1, hi - 2));
        double z0 = TT(hi, hi) + 0.75 * w;
        sh = 2.0 * z0;
        th = z0 * z0 + 0.4375 * w * w;
      } else {
        sh = TT(p, p) + TT(p + 1, p + 1);
        th = TT(p, p) * TT(p + 1, p + 1) - TT(p, p + 1) * TT(p + 1, p);
      }
    }
    q_acquire(Q, lane);
    if (*Q.err) { status = 2; break; }
    Refl* rl = Q.refl(Q.bq);
    const int rounds = (hi - 1 - l) + kBulgeGap * (nb - 1) + 1;
    for (int t = 0; t < rounds; ++t) {
      const int kq = l + t - kBulgeGap * warp;
      const bool act = warp < nb && kq >= l && kq <= hi - 1;
      Refl r;
      r.tau = 0.0;
      r.n = 0;
      r.pos = kq;
      if (act) {
        int n = kq <= hi - 2 ? 3 : 2;
        double x, y, z;
        if (kq == l) {
          x = TT(l, l) * TT(l, l) + TT(l, l + 1) * TT(l + 1, l) - sh * TT(l, l) + th;
          y = TT(l + 1, l) * (TT(l, l) + TT(l + 1, l + 1) - sh);
          z = n == 3 ? TT(l + 1, l) * TT(l + 2, l + 1) : 0.0;
        } else {
          x = TT(kq, kq - 1);
          y = TT(kq + 1, kq - 1);
          z = n == 3 ? TT(kq + 2, kq - 1) : 0.0;
        }
        make_refl(x, y, z, n, r);
        r.pos = kq;
        if (r.n != 0)
          for (int i = l + wl; i <= min(kq + 3, hi); i += 32) refl_row(S.T, S.ld, r, i);
      }
      if (warp < nb && wl == 0) rl[t * nb + warp] = r;
      __syncthreads();
      if (act) {
        int c0 = kq > l ? kq - 1 : l;
        if (r.n != 0)
          for (int c = c0 + wl; c <= hi; c += 32) refl_col(S.T, S.ld, r, c);
        if (kq > l && wl == 0) {
          TT(kq + 1, kq - 1) = 0.0;
          if (r.n == 3) TT(kq + 2, kq - 1) = 0.0;
        }
      }
      __syncthreads();
    }
    q_publish(Q, lane, 1, l, hi, nb, rounds, 0);
  }
  // last batch (with any pending rotations), then wait until both helpers
  // have applied everything and written Z back
  q_acquire(Q, lane);
  q_publish(Q, lane, 0, 0, 0, 0, 0, 1);
  if (lane == 0 && !mbar_wait_cluster(&Q.bars[4], 0, Q.limit)) *Q.err = 1;
  __syncthreads();
  if (*Q.err) status = 2;
  sweeps = total;
  return status;
}

// A helper's copy of a reflector, rescaled to a unit leading entry:
// P = I - tau u u^T = I - tv v v^T with v = u / u_0, tv = tau u_0^2, and
// w = tv v, so that applying P to a 3-vector a is s = a_0 + v_1 a_1 + v_2 a_2,
// a -= s [tv, w_1, w_2]: five FP64 instructions instead of seven.  (The Ritz
// CTA keeps the u form: there the product u^T a can start before tau is
// known, which shortens the latency chain of each bulge-chase round.)
struct alignas(16) HRefl {
  double v1, v2, tv, w1, w2;
  int pos, n;   // n = 0: skip
};
static_assert(sizeof(HRefl) == sizeof(Refl), "a helper's copy reuses the batch layout");

// Applies the reflectors rl[0..nref) in order to the strided vector x[k st]
// (a row of a column-major matrix when st = ld, a column when st = 1), each
// to its entries pos..pos+n-1; entries with n = 0 are skipped.  The next
// reflector's entries are loaded before the current one is applied, so that
// the load latency (distributed shared memory for the T helper) overlaps the
// FP64 chain; an entry that both touch is taken from the registers.
__device__ void apply_seq(double* x, int st, const HRefl* rl, int nref) {
  int t = 0;
  while (t < nref && rl[t].n == 0) ++t;
  if (t >= nref) return;
  HRefl r = rl[t];
  double a0 = x[r.pos * st], a1 = x[(r.pos + 1) * st], a2 = r.n == 3 ? x[(r.pos + 2) * st] : 0.0;
  for (;;) {
    int tn = t + 1;
    while (tn < nref && rl[tn].n == 0) ++tn;
    const bool more = tn < nref;
    HRefl q;
    double b0 = 0.0, b1 = 0.0, b2 = 0.0;
    if (more) {
      q = rl[tn];
      b0 = x[q.pos * st];
      b1 = x[(q.pos + 1) * st];
      if (q.n == 3) b2 = x[(q.pos + 2) * st];
    }
    double sd = fma(r.v1, a1, a0);
    if (r.n == 3) sd = fma(r.v2, a2, sd);
    a0 = fma(-r.tv, sd, a0);
    a1 = fma(-r.w1, sd, a1);
    x[r.pos * st] = a0;
    x[(r.pos + 1) * st] = a1;
    if (r.n == 3) {
      a2 = fma(-r.w2, sd, a2);
      x[(r.pos + 2) * st] = a2;
    }
    if (!more) return;
    // q's entry k is r's entry k + d
    const int d = q.pos - r.pos;
    b0 = d == 0 ? a0 : d == 1 ? a1 : (d == 2 && r.n == 3) ? a2 : b0;
    b1 = d == -1 ? a0 : d == 0 ? a1 : (d == 1 && r.n == 3) ? a2 : b1;
    b2 = d == -2 ? a0 : d == -1 ? a1 : (d == 0 && r.n == 3) ? a2 : b2;
    a0 = b0;
    a1 = b1;
    a2 = b2;
    r = q;
    t = tn;
  }
}

// Helper CTA (cluster rank 1: Z, rank 2: T outside the window) of the QR
// iteration: takes the batches in order, copies each into its own shared
// memory (releasing the buffer), and applies it.  Rank 1 copies Z from the
// Ritz CTA before the first batch and writes it back after the last.
__device__ void ritz_helper(const RitzArgs& R, unsigned rank, Smem& S, Queue& Q) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int m = R.m, ld = S.ld, lane = threadIdx.x;
  const int maxref = kBulges * (m + 4 * kBulges);
  const char* rbuf = cl.map_shared_rank(Q.buf, 0);
  double* T0 = cl.map_shared_rank(S.T, 0);
  double* Z0 = cl.map_shared_rank(S.Z, 0);
  Rot* lrot = Q.rot(0);     // this CTA's copy of the current batch
  HRefl* lrl = (HRefl*)Q.refl(0);   // same size as Refl
  // rank 2 works on its own copy of the entries outside the window: taken
  // from the Ritz CTA when a batch first touches them (own = 1), written
  // back at the end; its T and Z areas hold the copy and the flags
  double* Tl = S.T;
  unsigned char* own = (unsigned char*)S.Z;
  if (rank == 2)
    for (int e = lane; e < ld * m; e += NT) own[e] = 0;
  int err = 0;
  for (int b = 0;; ++b) {
    if (lane == 0)
      *Q.err = mbar_wait_cluster(&Q.bars[b & 1], (uint32_t)((b >> 1) & 1), Q.limit) ? 0 : 1;
    __syncthreads();
    if (*Q.err) { err = 1; break; }
    fence_acq_rel_cluster();
    const char* src = rbuf + (size_t)(b & 1) * Q.bbytes;
    const BatchHdr h = *(const BatchHdr*)src;
    // entries are checked against the matrix so that no access can leave it
    const int nrot = min(max(h.nrot, 0), kMaxRot);
    const int nref = h.sweep ? min(max(h.rounds * h.nb, 0), maxref) : 0;
    const int l = min(max(h.l, 0), m - 1), hi = min(max(h.hi, l), m - 1);
    for (int q = lane; q < nrot; q += NT) {
      Rot rt = ((const Rot*)(src + sizeof(BatchHdr)))[q];
      if (rt.j < 0 || rt.j > m - 2) { rt.c = 1.0; rt.s = 0.0; rt.j = 0; }
      lrot[q] = rt;
    }
    for (int q = lane; q < nref; q += NT) {
      const Refl r = ((const Refl*)(src + kReflOff))[q];
      HRefl hr;
      // n = 0 marks an entry to skip: an inactive bulge, a zero reflector,
      // or (never in a correct batch) one that would leave the matrix.
      // A nonzero reflector has |u_0| = |x_0| + ||x|| > 0.
      if (r.n < 2 || r.n > 3 || r.pos < 0 || r.pos + r.n > m || !(r.tau != 0.0) || !(r.u0 != 0.0)) {
        hr.v1 = hr.v2 = hr.tv = hr.w1 = hr.w2 = 0.0;
        hr.n = 0;
        hr.pos = 0;
      } else {
        const double ru = 1.0 / r.u0;
        hr.v1 = r.u1 * ru;
        hr.v2 = r.n == 3 ? r.u2 * ru : 0.0;
        hr.tv = r.tau * r.u0 * r.u0;
        hr.w1 = hr.tv * hr.v1;
        hr.w2 = hr.tv * hr.v2;
        hr.n = r.n;
        hr.pos = r.pos;
      }
      lrl[q] = hr;
    }
    if (rank == 1 && b == 0)
      for (int i = lane; i < ld * m; i += NT) S.Z[i] = Z0[i];
    __syncthreads();
    if (lane == 0) mbar_arrive_remote(&Q.bars[2 + (b & 1)], 0);
    if (rank == 1) {
      // Z <- Z G for each rotation, then Z <- Z P for each reflector; one row per thread
      for (int i = lane; i < m; i += NT) {
        for (int q = 0; q < nrot; ++q) {
          const int j = lrot[q].j;
          const double c = lrot[q].c, sn = lrot[q].s;
          double a = S.Z[i + ld * j], bb = S.Z[i + ld * (j + 1)];
          S.Z[i + ld * j] = c * a + sn * bb;
          S.Z[i + ld * (j + 1)] = -sn * a + c * bb;
        }
        apply_seq(S.Z + i, ld, lrl, nref);
      }
    } else {
      // take over the entries this batch touches that the Ritz CTA has not
      // handed over yet (they never return to its window)
      for (int q = 0; q < nrot; ++q) {
        const int j = lrot[q].j, nc = m - j - 2;
        for (int u = lane; u < nc + j; u += NT) {
          const int e = u < nc ? j + ld * (j + 2 + u) : (u - nc) + ld * j;
          const int e2 = u < nc ? e + 1 : e + ld;
          if (!own[e]) { Tl[e] = T0[e]; own[e] = 1; }
          if (!own[e2]) { Tl[e2] = T0[e2]; own[e2] = 1; }
        }
      }
      if (h.sweep) {
        const int nw = hi - l + 1;
        const int cr = l * nw, cc = nw * (m - 1 - hi);
        for (int u = lane; u < cr + cc; u += NT) {
          const int e = u < cr ? (u % l) + ld * (l + u / l)
                               : (l + (u - cr) % nw) + ld * (hi + 1 + (u - cr) / nw);
          if (!own[e]) { Tl[e] = T0[e]; own[e] = 1; }
        }
      }
      __syncthreads();
      // rotations: rows j, j+1 right of the block (from the left), columns
      // j, j+1 above it (from the right)
      for (int q = 0; q < nrot; ++q) {
        const int j = lrot[q].j;
        const double c = lrot[q].c, sn = lrot[q].s;
        const int nc = m - j - 2;
        for (int u = lane; u < nc + j; u += NT) {
          double *pa, *pb;
          if (u < nc) {
            const int col = j + 2 + u;
            pa = Tl + j + ld * col;
            pb = pa + 1;
          } else {
            pa = Tl + (u - nc) + ld * j;
            pb = pa + ld;
          }
          double a = *pa, bb = *pb;
          *pa = c * a + sn * bb;
          *pb = -sn * a + c * bb;
        }
        __syncthreads();
      }
      // the sweep: columns right of the window (rows l..hi, from the left)
      // and rows above it (columns l..hi, from the right)
      const int ncol = m - 1 - hi, nrow = l;
      for (int u = lane; u < ncol + nrow; u += NT) {
        if (u < ncol)
          apply_seq(Tl + ld * (hi + 1 + u), 1, lrl, nref);
        else
          apply_seq(Tl + (u - ncol), ld, lrl, nref);
      }
    }
    __syncthreads();
    if (h.end) break;
  }
  if (rank == 1 && !err)
    for (int i = lane; i < ld * m; i += NT) Z0[i] = S.Z[i];
  if (rank == 2 && !err)
    for (int e = lane; e < ld * m; e += NT)
      if (own[e]) T0[e] = Tl[e];
  fence_acq_rel_cluster();
  __syncthreads();
  if (lane == 0) {
    if (err) *cl.map_shared_rank(Q.err, 0) = 1;
    fence_acq_rel_cluster();
    mbar_arrive_remote(&Q.bars[4], 0);
  }
}

__device__ void hessenberg(Smem& S, int m, int lane, int lock) {
  for (int c = lock; c + 2 < m; ++c) {
    int n = m - c - 1;
    // Householder vector of T[c+1:m, c]; computed redundantly
    double alpha = TT(c + 1, c), sg = 0.0;
    for (int i = 1 + lane; i < n; i += NT) sg += TT(c + 1 + i, c) * TT(c + 1 + i, c);
    sg = block_sum(sg, S.red, lane);
    if (sg == 0.0) continue;
    double nr = sqrt_nr(alpha * alpha + sg);
    double beta = alpha <= 0.0 ? nr : -nr;
    double d = alpha - beta;
    double tau = div_nr(beta - alpha, beta);
    double rd = rcp_nr(d);
    __syncthreads();
    for (int i = lane; i < n; i += NT) S.v[i] = i == 0 ? 1.0 : TT(c + 1 + i, c) * rd;
    __syncthreads();
    apply_left(S.T, S.ld, S.v, tau, n, c + 1, c, m, lane);
    __syncthreads();
    apply_right_tz(S.T, S.Z, m, S.ld, S.v, tau, n, c + 1, 0, m, lane);
    __syncthreads();
    if (lane == 0)
      for (int i = 1; i < n; ++i) TT(c + 1 + i, c) = 0.0;
    __syncthreads();
  }
}

__device__ inline void cdiv(double ar, double ai, double br, double bi, double& cr, double& ci) {
  // (ar + i ai) / (br + i bi), scaled by the larger of |br|, |bi| (Smith)
  if (fabs(br) >= fabs(bi)) {
    double r = bi * rcp_nr(br), d = rcp_nr(br + bi * r);
    cr = (ar + ai * r) * d;
    ci = (ai - ar * r) * d;
  } else {
    double r = br * rcp_nr(bi), d = rcp_nr(bi + br * r);
    cr = (ar * r + ai) * d;
    ci = (ai * r - ar) * d;
  }
}

// Per-warp buffers of the eigenvector back substitution (6 vectors of m).
struct WarpVec {
  double *yr, *yi, *sr, *si, *dr, *di;
};

// Eigenvector y of the quasi-triangular T for the eigenvalue at diagonal
// position j (lr, li; li > 0 means j starts its 2 x 2 block), computed by one
// warp: y = e_j (or the block's null vector) above which rows are solved
// from the bottom up, (T_ii - lambda) y_i = -sum_{c>i} T_ic y_c, with the reciprocals of the
// diagonal 1 x 1 shifts T_ii - lambda and of the 2 x 2 block determinants
// formed first, in parallel over the lanes, so that the sequential chain per
// row is a complex multiply and a residual update.
__device__ void trevc_warp(const double* T, int m, int ld, int j, double lr, double li,
                           double smin, const double* wi, int wl, WarpVec& B) {
  const bool pair = (li != 0.0);
  for (int i = wl; i < m; i += 32) { B.yr[i] = 0.0; B.yi[i] = 0.0; }
  __syncwarp();
  int top;
  if (!pair) {
    if (wl == 0) B.yr[j] = 1.0;
    top = j;
  } else {
    if (wl == 0) {
      B.yr[j] = T[j + ld * (j + 1)];
      B.yi[j] = 0.0;
      B.yr[j + 1] = lr - T[j + ld * j];
      B.yi[j + 1] = li;
    }
    top = j + 1;
  }
  __syncwarp();
  for (int r = wl; r < j; r += 32) {
    double ar = 0.0, ai = 0.0;
    for (int l = j; l <= top; ++l) { ar -= T[r + ld * l] * B.yr[l]; ai -= T[r + ld * l] * B.yi[l]; }
    B.sr[r] = ar;
    B.si[r] = ai;
    // reciprocal of the shifted diagonal (1 x 1 rows) or of the determinant of
    // the shifted 2 x 2 block (stored at its first row)
    if (wi[r] == 0.0) {
      double dr = T[r + ld * r] - lr, di = -li;
      if (fabs(dr) + fabs(di) < smin) dr = smin;
      cdiv(1.0, 0.0, dr, di, B.dr[r], B.di[r]);
    } else if (wi[r] > 0.0) {
      int i0 = r, i1 = r + 1;
      double ar2 = T[i0 + ld * i0] - lr, ai2 = -li, br = T[i0 + ld * i1], cr = T[i1 + ld * i0];
      double dr = T[i1 + ld * i1] - lr, di = -li;
      double detr = ar2 * dr - ai2 * di - br * cr, deti = ar2 * di + ai2 * dr;
      if (fabs(detr) + fabs(deti) < smin) detr = smin;
      cdiv(1.0, 0.0, detr, deti, B.dr[r], B.di[r]);
    }
  }
  __syncwarp();
  int i = j - 1;
  while (i >= 0) {
    if (wi[i] >= 0.0) {   // 1 x 1 row
      double s_r = B.sr[i], s_i = B.si[i], pr = B.dr[i], pi = B.di[i];
      double yr = s_r * pr - s_i * pi, yi = s_r * pi + s_i * pr;
      if (wl == 0) { B.yr[i] = yr; B.yi[i] = yi; }
      for (int r = wl; r < i; r += 32) {
        B.sr[r] -= T[r + ld * i] * yr;
        B.si[r] -= T[r + ld * i] * yi;
      }
      __syncwarp();
      i -= 1;
    } else {              // rows i-1, i form a 2 x 2 block
      int i0 = i - 1;
      double ar = T[i0 + ld * i0] - lr, ai = -li, br = T[i0 + ld * i], cr = T[i + ld * i0];
      double dr = T[i + ld * i] - lr, di = -li;
      double s0r = B.sr[i0], s0i = B.si[i0], s1r = B.sr[i], s1i = B.si[i];
      double n0r = s0r * dr - s0i * di - br * s1r, n0i = s0r * di + s0i * dr - br * s1i;
      double n1r = ar * s1r - ai * s1i - cr * s0r, n1i = ar * s1i + ai * s1r - cr * s0i;
      double pr = B.dr[i0], pi = B.di[i0];
      double y0r = n0r * pr - n0i * pi, y0i = n0r * pi + n0i * pr;
      double y1r = n1r * pr - n1i * pi, y1i = n1r * pi + n1i * pr;
      if (wl == 0) { B.yr[i0] = y0r; B.yi[i0] = y0i; B.yr[i] = y1r; B.yi[i] = y1i; }
      for (int r = wl; r < i0; r += 32) {
        B.sr[r] -= T[r + ld * i0] * y0r + T[r + ld * i] * y1r;
        B.si[r] -= T[r + ld * i0] * y0i + T[r + ld * i] * y1i;
      }
      __syncwarp();
      i -= 2;
    }
  }
  __syncwarp();
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Shared-memory layout, the same in every CTA of the cluster (the helpers
// address the Ritz CTA's T, Z and batches at their own offsets).
__device__ void ritz_layout(double* sm, int m, Smem& S, double*& wbuf, int*& wlist) {
  S.ld = m | 1;
  S.T = sm;
  S.Z = S.T + S.ld * m;
  S.v = S.Z + S.ld * m;
  S.wr = S.v + m;
  S.wi = S.wr + m;
  S.red = S.wi + m;
  S.rank = (int*)(S.red + NT / 32);
  S.sel = S.rank + m;
  S.cflag = S.sel + m;
  S.batch = (char*)(((uintptr_t)(S.cflag + m) + 15) & ~(uintptr_t)15);
  wbuf = (double*)(S.batch + 2 * batch_bytes(m));
  wlist = (int*)(wbuf + 6 * kVecWarps * m);
}

// The Ritz CTA (cluster rank 0): steps 1-6.
__device__ void ritz_main(const RitzArgs& R, Smem& S, Queue& Q, double* wbuf, int* wlist) {
  const int m = R.m;
  const int lane = threadIdx.x;  // thread index in the CTA
  const int warp = lane >> 5, wl = lane & 31;
  const int vw = warp < kVecWarps ? warp : 0;
  WarpVec B{wbuf + 6 * m * vw,         wbuf + 6 * m * vw + m, wbuf + 6 * m * vw + 2 * m,
            wbuf + 6 * m * vw + 3 * m, wbuf + 6 * m * vw + 4 * m, wbuf + 6 * m * vw + 5 * m};
  __shared__ int wcount[NT / 32];

  for (int i = lane; i < S.ld * m; i += NT) {
    int r = i % S.ld, c = i / S.ld;
    S.T[i] = r < m ? R.H[r + (m + 1) * c] : 0.0;
    S.Z[i] = (r == c) ? 1.0 : 0.0;
  }
  const double beta = R.H[m + (m + 1) * (m - 1)];
  __syncthreads();
  long long t_ph[7];
  t_ph[0] = clock64();
  hessenberg(S, m, lane, R.lock);
  t_ph[1] = clock64();
  int sweeps = 0;
  const int qr_status = francis(S, m, lane, sweeps, R.lock, Q);
  t_ph[2] = clock64();
  __syncthreads();
  if (qr_status == 2) {   // the helpers' results are incomplete: report and stop
    if (lane == 0) {
      R.out->fail = 2;
      R.out->finished = 1;
      R.out->sweeps = sweeps;
    }
    return;
  }
  const bool ok = qr_status == 0;
  // eigenvalues in Schur order
  if (lane == 0) {
    int pos = 0;
    while (pos < m) {
      if (pos + 1 < m && TT(pos + 1, pos) != 0.0) {
        double a = TT(pos, pos), im = sqrt(fabs(TT(pos, pos + 1) * TT(pos + 1, pos)));
        S.wr[pos] = a; S.wi[pos] = im;
        S.wr[pos + 1] = a; S.wi[pos + 1] = -im;
        pos += 2;
      } else {
        S.wr[pos] = TT(pos, pos);
        S.wi[pos] = 0.0;
        pos += 1;
      }
    }
  }
  __syncthreads();
  // ranks by |lambda - s| = 1/|theta|, Im lambda > 0 first on ties
  // (lambda - s = 1/theta, so Im lambda has the sign of -Im theta)
  // |lambda - s| = 1/|theta|: nearer means larger |theta|^2
  // |theta|^2 of every position (S.v is free after the QR) and its class
  // (Im theta < 0, = 0, > 0) in S.cflag (reset below); the comparisons are
  // then integer ones: non-negative doubles order as their bit patterns
  for (int i = lane; i < m; i += NT) {
    S.v[i] = S.wr[i] * S.wr[i] + S.wi[i] * S.wi[i];
    const long long b = __double_as_longlong(S.wi[i]);
    S.cflag[i] = (b << 1) == 0 ? 1 : (b < 0 ? 0 : 2);
  }
  __syncthreads();
  for (int i = lane; i < m; i += NT) {
    const long long ti = __double_as_longlong(S.v[i]);
    const int ci = S.cflag[i];
    int rk = 0;
    for (int q = 0; q < m; ++q) {
      const long long tq = __double_as_longlong(S.v[q]);
      const int cq = S.cflag[q];
      if (tq > ti || (tq == ti && (cq < ci || (cq == ci && q < i)))) ++rk;
    }
    S.rank[i] = rk;
  }
  __syncthreads();
  double tnorm = frob(S, m, lane);
  double smin = fmax(kEps * tnorm, 1e-300);
  t_ph[3] = clock64();
  for (int i = lane; i < m; i += NT) S.cflag[i] = 0;
  __syncthreads();
  // wanted pairs: eigenvectors, estimates and (when finishing) the outputs.
  // final_pass 1 always finishes; 2 finishes when every wanted pair has
  // converged (the restart is then not needed), else restarts.
  bool fin = R.final_pass == 1;
  int nconv = 0;
  // wanted positions in Schur order; each warp takes every fourth one
  if (lane == 0) {
    int c = 0;
    for (int pos = 0; pos < m; ++pos)
      if (S.rank[pos] < R.neig) wlist[c++] = pos;
    wcount[0] = c;
  }
  __syncthreads();
  const int nwant = wcount[0];
  __syncthreads();
  for (int attempt = 0; attempt < 2; ++attempt) {
    int myconv = 0;
    for (int e = warp; warp < kVecWarps && e < nwant; e += kVecWarps) {
      const int pos = wlist[e];
      const int rk = S.rank[pos];
      if (!fin && pos < R.lock) {
        // locked: converged and decoupled, its estimate is zero
        ++myconv;
        if (wl == 0) {
          double ir, ii;
          cdiv(1.0, 0.0, S.wr[pos], S.wi[pos], ir, ii);
          R.out->lam[2 * rk] = R.sigma + R.tscale * ir;
          R.out->lam[2 * rk + 1] = R.tscale * ii;
          R.out->est[rk] = 0.0;
          S.cflag[pos] = 1;
        }
        continue;
      }
      double lr = S.wr[pos], li = S.wi[pos];
      int jstart = (li < 0.0) ? pos - 1 : pos;   // conjugate: start of its block
      trevc_warp(S.T, m, S.ld, jstart, lr, fabs(li), smin, S.wi, wl, B);
      // y_H = Z y ; estimate uses the last row; norm of y equals norm of Z y
      double nrm = 0.0, lastr = 0.0, lasti = 0.0;
      for (int l = wl; l < m; l += 32) {
        nrm += B.yr[l] * B.yr[l] + B.yi[l] * B.yi[l];
        lastr += ZZ(m - 1, l) * B.yr[l];
        lasti += ZZ(m - 1, l) * B.yi[l];
      }
      nrm = sqrt(warp_sum(nrm));
      lastr = warp_sum(lastr);
      lasti = warp_sum(lasti);
      double theta = hypot(lr, li);
      double est = fabs(beta) * hypot(lastr, lasti) / (nrm * theta);
      if (est <= R.tol) ++myconv;
      if (wl == 0) {
        S.cflag[pos] = est <= R.tol ? 1 : 0;
        // lambda = s + 1/theta
        double ir, ii;
        cdiv(1.0, 0.0, lr, li, ir, ii);
        R.out->lam[2 * rk] = R.sigma + R.tscale * ir;
        R.out->lam[2 * rk + 1] = R.tscale * ii;
        R.out->est[rk] = est;
      }
      if (fin) {
        double sgn = (li < 0.0) ? -1.0 : 1.0;
        for (int r = wl; r < m; r += 32) {
          double ar = 0.0, ai = 0.0;
          for (int l = 0; l < m; ++l) { ar += ZZ(r, l) * B.yr[l]; ai += ZZ(r, l) * B.yi[l]; }
          R.Y[2 * (r + m * rk)] = ar / nrm;
          R.Y[2 * (r + m * rk) + 1] = sgn * ai / nrm;
        }
      }
      __syncwarp();
    }
    if (wl == 0) wcount[warp] = myconv;
    __syncthreads();
    nconv = 0;
    for (int w = 0; w < kVecWarps; ++w) nconv += wcount[w];
    __syncthreads();
    if (fin || R.final_pass != 2 || nconv < R.neig) break;
    fin = true;
    __syncthreads();
  }
  t_ph[4] = clock64();
  if (lane == 0) {
    R.out->n_conv = nconv;
    R.out->fail = ok ? 0 : 1;
    R.out->beta = beta;
    R.out->sweeps = sweeps;
    R.out->finished = fin ? 1 : 0;
    if (fin) {
      for (int q = 0; q < 4; ++q) R.out->phase_cycles[q] = t_ph[q + 1] - t_ph[q];
      R.out->phase_cycles[4] = R.out->phase_cycles[5] = 0;
    }
  }
  if (fin) return;
  // select the kwant nearest, never splitting a conjugate pair
  // locked blocks always stay (they sit at the top with a zero spike)
  for (int i = lane; i < m; i += NT) S.sel[i] = (S.rank[i] < R.kwant || i < R.lock) ? 1 : 0;
  __syncthreads();
  if (lane == 0) {
    int pos = 0;
    while (pos < m) {
      if (pos + 1 < m && TT(pos + 1, pos) != 0.0) {
        int s = S.sel[pos] | S.sel[pos + 1];
        S.sel[pos] = s;
        S.sel[pos + 1] = s;
        pos += 2;
      } else {
        pos += 1;
      }
    }
  }
  __syncthreads();
  // reorder: move selected blocks to the top
  const int k = reorder_parallel(S, m, tnorm, lane);
  __syncthreads();
  t_ph[5] = clock64();
  // locking: converged blocks among the kept ones move to the front (after
  // the blocks locked earlier); their spike entries are dropped below, which
  // decouples them from the rest of the projected matrix
  int nl = R.lock;
  int pos = R.lock;
  while (pos < k) {
    int bs = (pos + 1 < m && TT(pos + 1, pos) != 0.0) ? 2 : 1;
    bool conv = S.cflag[pos] && (bs == 1 || S.cflag[pos + 1]);
    if (conv) {
      int here = pos;
      while (here > nl) {
        int nbf = (here >= 2 && TT(here - 1, here - 2) != 0.0) ? 2 : 1;
        int prev = here - nbf;
        int cf_oth[2] = {S.cflag[prev], nbf == 2 ? S.cflag[prev + 1] : 0};
        __syncthreads();
        swap_blocks(S, m, prev, nbf, bs, tnorm, lane);
        __syncthreads();
        if (lane == 0) {
          for (int i = 0; i < bs; ++i) S.cflag[prev + i] = 1;
          for (int i = 0; i < nbf; ++i) S.cflag[prev + bs + i] = cf_oth[i];
        }
        __syncthreads();
        here = prev;
      }
      nl += bs;
    }
    pos += bs;
  }
  __syncthreads();
  for (int i = lane; i < (m + 1) * m; i += NT) {
    int r = i % (m + 1), c = i / (m + 1);
    double v = 0.0;
    if (c < k) {
      if (r < k) v = TT(r, c);
      else if (r == k && c >= nl) v = beta * ZZ(m - 1, c);
    }
    R.Hnew[i] = v;
  }
  for (int i = lane; i < m * k; i += NT) R.Q[i] = ZZ(i % m, i / m);
  if (lane == 0) {
    R.out->k = k;
    R.out->n_lock = nl;
    t_ph[6] = clock64();
    for (int q = 0; q < 6; ++q) R.out->phase_cycles[q] = t_ph[q + 1] - t_ph[q];
  }
}

// One cluster of kRitzCTAs CTAs.  Every wait inside is bounded except the
// two cluster barriers, which every CTA reaches on every path.
__global__ void __launch_bounds__(NT) k_ritz(RitzArgs R) {
  extern __shared__ double sm[];
  __shared__ uint64_t qbar[5];
  __shared__ int qerr;
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const unsigned rank = cl.block_rank();
  if (threadIdx.x == 0) {
    qerr = 0;
    mbar_init(&qbar[0], 1);                 // full: the Ritz CTA arrives
    mbar_init(&qbar[1], 1);
    for (int i = 2; i < 5; ++i) mbar_init(&qbar[i], kRitzCTAs - 1);   // empty, done: each helper
    mbar_fence_init();
  }
  cl.sync();   // every barrier is initialised before any CTA arrives on it
  Smem S;
  double* wbuf;
  int* wlist;
  ritz_layout(sm, R.m, S, wbuf, wlist);
  Queue Q{S.batch, batch_bytes(R.m), qbar, &qerr, R.wait_limit, 0, 0, false};
  if (rank == 0)
    ritz_main(R, S, Q, wbuf, wlist);
  else
    ritz_helper(R, rank, S, Q);
  cl.sync();   // no CTA leaves while another may still address its shared memory
}

}  // namespace

size_t ritz_smem(int m) {
  return sizeof(double) * (2 * (size_t)(m | 1) * m + 4 * (size_t)m + NT / 32) + 3 * sizeof(int) * m + 16 +
         2 * batch_bytes(m) + sizeof(double) * 6 * kVecWarps * (size_t)m + sizeof(int) * (size_t)m;
}

void launch_ritz(const double* H, double* Hnew, double* Q, double* Y, RitzOut* out, int m, int neig,
                 int kwant, int final_pass, int lock, double sigma, double tol, double tscale,
                 cudaStream_t s) {
  RitzArgs R{H, Hnew, Q, Y, out, m, neig, kwant, final_pass, lock, sigma, tol, ritz_wait_limit(),
             tscale};
  size_t smem = ritz_smem(m);
  smem_at_least((const void*)k_ritz, smem);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kRitzCTAs);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kRitzCTAs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  RQ_CUDA(cudaLaunchKernelEx(&cfg, k_ritz, R));
}

}  // namespace rq
