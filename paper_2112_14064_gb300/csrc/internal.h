// Internal declarations shared by the CUDA translation units of rigaqep.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <stdexcept>
#include <string>
#include <utility>
#include <vector>

#include "../../include/rigaqep.h"
#include "plan.h"

namespace rq {

constexpr int kMaxKrylov = 96;   // largest Krylov dimension m
constexpr int kMaxP = 8;         // largest B-spline degree

// Error carried through the C++ layers and mapped to a status at the ABI.
struct Error : std::runtime_error {
  rigaqep_status code;
  Error(rigaqep_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define RQ_CUDA(call)                                                                     \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      throw ::rq::Error(e_ == cudaErrorMemoryAllocation ? RIGAQEP_ERR_OOM : RIGAQEP_ERR_CUDA, \
                        std::string(#call) + ": " + cudaGetErrorString(e_));              \
  } while (0)

// Stream-ordered allocation.  Device buffers come from a library-owned memory
// pool of the current device (cudaMallocFromPoolAsync / cudaFreeAsync), so
// that allocating and releasing never synchronises the device: handles that
// run on different streams (a batch) do not serialise each other, and
// repeated solves reuse the pool's memory.  Allocations are ordered on the
// stream of the entry point that is running (set by StreamScope); a buffer is
// released on the stream it was allocated on, so that stream must outlive it.
cudaMemPool_t device_pool();
inline thread_local cudaStream_t t_stream = nullptr;
struct StreamScope {
  cudaStream_t old;
  explicit StreamScope(cudaStream_t s) : old(t_stream) { t_stream = s; }
  ~StreamScope() { t_stream = old; }
};

// Programmatic dependent launch for the kernels of the operator and
// Gram-Schmidt chain: a kernel launched this way may start while the previous
// kernel of the stream drains.  Such a kernel calls pdl_trigger() first (its
// own dependents may then launch once all its blocks have started) and
// pdl_wait() before it reads anything an earlier kernel of the stream wrote
// (the wait returns when the previous kernel has completed and its memory is
// visible; it is a no-op for an ordinary launch).
template <class... KArgs, class... Args>
void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  RQ_CUDA(cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...));
}
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
#endif

// Polls after which a wait between the CTAs of the Ritz step gives up
// (process-wide; rigaqep_set_wait_limit).
constexpr uint32_t kDefaultWaitLimit = 1u << 22;
uint32_t ritz_wait_limit();
void set_ritz_wait_limit(uint32_t polls);

// Raises a kernel's dynamic shared memory limit to at least `bytes` (never
// lowers it, so concurrent callers with different sizes cannot race a launch
// below its own request).
void smem_at_least(const void* kernel, size_t bytes);

// Owning device buffer.
template <class T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  cudaStream_t st = nullptr;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() { release(); }
  void release() {
    if (p) cudaFreeAsync(p, st);
    p = nullptr;
    n = 0;
  }
  void alloc(size_t count) {
    release();
    if (count == 0) count = 1;
    st = t_stream;
    RQ_CUDA(cudaMallocFromPoolAsync((void**)&p, count * sizeof(T), device_pool(), st));
    n = count;
  }
  template <class A>
  void upload(const std::vector<T, A>& h, cudaStream_t s) {
    alloc(h.size());
    if (!h.empty()) RQ_CUDA(cudaMemcpyAsync(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  }
};

// Device-side status word written by kernels instead of trapping.
struct DevStatus {
  int32_t pivot_fail;   // first failing supernode + 1 (0 = none)
  int32_t ritz_fail;    // QR iteration limit reached
  int32_t internal;     // consistency check failed
  int32_t timeout;      // a bounded wait ran out (1: tensor-core pipeline, 2: FB items)
  int32_t neg_pivots;   // negative pivots of an indefinite factorisation (inertia)
  int32_t pad[3];
};

// Output of the Ritz kernel.
struct RitzOut {
  int32_t n_conv;       // wanted pairs (first neig) with estimate <= tol
  int32_t k;            // kept dimension after reordering (restart)
  int32_t fail;         // 1: QR did not converge, 2: a bounded wait between the CTAs ran out
  int32_t sweeps;       // Francis double-shift sweeps of this step
  int32_t n_lock;       // leading Schur columns locked after this restart
  int32_t finished;     // eigenvectors written, no restart data
  double beta;
  long long phase_cycles[6];     // hessenberg, QR, eigenvalues+ranks, eigvecs, reorder, lock
  double lam[2 * kMaxKrylov];    // wanted lambdas (re, im), first neig
  double est[kMaxKrylov];        // Ritz estimates of the wanted pairs
};

// Staged-operand geometry of one front for the tensor-core products
// (tcfront.cu): rows of the 128-byte K-block layout, counted from the start
// of the front's level region.
struct TcFront {
  int32_t u, k, kb, a;                  // update rows, pivots, K-blocks, first pivot
  int32_t offA3, offB3, offB5, offA4;   // F21, inv(L11) rows, inv(L11) columns, L21
  int32_t offB4, nB0, pad0, pad1;       // Z; B rows of the plain product
  int64_t loff, uoff;                   // FP32 panel and update-block offsets
};
static_assert(sizeof(TcFront) == 64, "TcFront layout");

// Plan and buffers of the tensor-core products of one precision.
struct TcPlan {
  bool ready = false, bf16 = false;
  DBuf<TcFront> fr;
  DBuf<int32_t> stage, t3, t3w, t45;    // stage items, tiles of (3) (N = 64, 128), of (4)+(5)
  std::vector<int32_t> stage_lvl, t3_lvl, t3w_lvl, t45_lvl;
  std::vector<int32_t> n35, kbmax;      // per level: N of product (3); K-blocks
  bool tuned = false;                   // n35 chosen by the autotuner (this or an earlier handle)
  std::vector<std::pair<float, float>> tune_ms;   // timings of N = 64 / 128 when tuned here
  DBuf<unsigned char> hi, lo;           // the two staged planes (split terms)
  DBuf<float> scale;                    // per-front power of two (BF16)
  CUtensorMap maps[4];                  // hi/lo planes, boxes of 128 and 64 rows
};

struct EigsParams {
  int neig;        // pairs returned
  int ncand;       // pairs converged around the shift
  double target;   // selection point
  double shift;    // spectral shift (Q factorised there)
  bool in_region;  // selection by target among the candidates
  int m, max_restarts;
  double tol;
  uint64_t seed;
  double vscale = 1.0;   // scaled pencil (Remark 4): lambda = vscale * gamma; 1 = unscaled
  // undamped pencil K x = mu M x (Lanczos): the basis keeps v_u = 0 and v_l = x,
  // the operator is (K - shift M)^{-1} M, the candidates in [lo, hi) are returned
  bool gep = false;
  double lo = 0.0, hi = 0.0;
  // complex shift s = shift + i shift_i (real operator Re((A - s B)^{-1} B);
  // the selection is nearest s)
  bool cplx = false;
  double shift_i = 0.0;
};

struct Problem {
  Plan plan;
  cudaStream_t stream = nullptr;
  int device = 0;               // CUDA device the handle was created on
  int nsm = 1;                  // its multiprocessor count (grid sizing)
  bool analyzed = false;
  bool factored = false;
  double fact_sigma = 0.0;
  rigaqep_info info{};

  // original-order CSR and values
  DBuf<int32_t> rowptr, col;
  DBuf<double> K, M, C;
  DBuf<double> sigma_e;
  DBuf<double> m1, k1;          // 1-D element mass / stiffness integrals
  DBuf<int> first_fn;           // first full function of each element
  // ND-ordered CSR and values
  DBuf<int32_t> rowptr_n, col_n, fpos;
  DBuf<int32_t> slot_map;
  DBuf<double> Kn, Mn, Cn;
  // the same pattern in SELL-32 (slices of 32 rows, each padded to its widest
  // row; entry k of row 32 s + l at sell_off[s] + 32 k + l) with M and C
  DBuf<int32_t> sell_off, sell_col;
  DBuf<double> sell_M, sell_C;
  std::vector<int32_t> sell_off_h;   // host copy (source of the upload)
  // symbolic on device
  DBuf<int32_t> perm, iperm, sptr, upd_ptr, upd_idx, relmap, child_ptr, child_idx, lvl_nodes;
  DBuf<int64_t> loff, uoff;
  // numeric factor
  DBuf<double> Lval, Uval, Dinv, Dval;
  // row panels of pivot blocks too wide for shared memory (16 rows x k per
  // item of such a level, any scalar type; sized in doubles)
  DBuf<double> panel_scratch;
  // pivot blocks wider than the cluster kernel: X_JJ and a rows x 32 buffer
  // per front of a level (sized in doubles for 16-byte scalars)
  DBuf<double> wide_scratch;
  int64_t wide_bstride = 32;
  // FP32 factor (mixed precision: FP32 fronts, FP64 iterative refinement)
  DBuf<float> Lval32, Uval32, Dinv32, Dval32, yvec32, zbuf32, ir_r32;
  DBuf<double> ir_y;
  bool fact_gep = false;        // the current factor is of K - fact_sigma M (undamped pencil)
  int gep_inside = 0;           // candidates inside the interval of the last undamped solve
  bool fact_fp32 = false;       // the current factor is stored in FP32 (FP32, TF32 or BF16 fronts)
  int32_t fact_prec = RIGAQEP_FP64;   // precision of the current factor
  TcPlan tc;                    // tensor-core products (TF32 / BF16 fronts)
  // complex-shift factor (complex FP64 scalars, 16 bytes each; cplx.cuh)
  struct Complex {
    DBuf<double2> Lval, Uval, Dinv, Dval, yvec, zbuf, y;
    DBuf<int32_t> piv_fronts;
    std::vector<int32_t> piv_lvl;
  } cx;
  bool fact_cplx = false;       // the current factor is the complex one (shift fact_sigma + i fact_sigma_i)
  double fact_sigma_i = 0.0;
  int n_ir = 0;                 // refinement steps per solve with the FP32 factor
  DBuf<int32_t> row_items, tile_items;    // factor work items (front, a, b, 0)
  DBuf<int32_t> piv_fronts;     // per level: small pivot blocks, then cluster-sized ones
  std::vector<int32_t> piv_lvl; // boundaries: level l small [3l, 3l+1), cluster [3l+1, 3l+2), wide [3l+2, 3l+3)
  std::vector<int32_t> row_lvl, tile_lvl;
  DBuf<double> yvec;            // FB update vectors (one per supernode, struct-sized)
  DBuf<double> xwork;           // FB work vector (N)
  DBuf<double> zbuf, wbuf;      // FB intermediates (N)
  DBuf<int32_t> fwd_items, bwd_items;   // FB work items (12 int32 each, see factor.cu)
  DBuf<int32_t> fb_gptr, fb_gsrc;       // per front position: children's update entries
  std::vector<int32_t> fwd_lvl, bwd_lvl;  // work items of each level
  std::vector<int32_t> fwd_rc;            // 32-row chunks per forward item, per level
  // dependency-driven sweeps of the upper levels (factor.cu)
  DBuf<int32_t> fb_parent, fb_kid_items, fb_bwd_items, fb_border;
  DBuf<unsigned> fb_counters;   // kdone[nsuper], bdone[nsuper], tickets[4]
  unsigned fb_epoch = 0;        // sweeps so far (the counters are cumulative)
  int dep_maxK = 1, dep_grid_fwd = 1, dep_grid_bwd = 1;
  // Krylov workspace
  DBuf<double> V, Vtmp, H, part, hvec, yop, wop, scal, Y;
  DBuf<RitzOut> ritz;
  DBuf<unsigned> counter;       // last-block-done counters of the fused reductions
  DBuf<DevStatus> status;
  int64_t Np = 0;               // N rounded up to 32
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double sigma_min = 0.0, sigma_max = 0.0;  // extremes of the damping coefficients
  double maxabs_K = 0.0, maxabs_M = 0.0;    // largest entries of K and M (scaling)
  int64_t launches = 0;         // kernel launches of the current call
  std::vector<int32_t> h_lvl_ptr;
  std::vector<int32_t> lvl_maxF;  // largest front order per level
  std::vector<int32_t> lvl_maxK;
  // converged candidates of the last in-region eigensolve (seeded start),
  // valid until the factor changes
  bool cand_valid = false;
  RitzOut cand{};
  EigsParams cand_E{};
  ~Problem();
};

// kernels / launch helpers (each .cu file)
void launch_assemble(Problem& P);
// ND-ordered CSR columns, original slots and front rows (after the symbolic
// arrays are on the device); err receives 1 or 2 on a bad pattern
void launch_nd_csr(Problem& P, int32_t* err);
void launch_permute_values(Problem& P);
// SELL-32 copy of the ND pattern with M and C (after launch_permute_values)
void launch_sell(Problem& P);
void launch_norms(Problem& P);
// precision: RIGAQEP_FP64, RIGAQEP_FP32_IR, RIGAQEP_TF32_IR or RIGAQEP_BF16_IR
void launch_factor(Problem& P, double sigma, int precision);
// LDL^T of K - mu M in FP64 with pivots of either sign (the undamped
// pencil's spectrum slicing): status->neg_pivots counts the negative ones
void launch_factor_gep(Problem& P, double mu);
// complex symmetric LDL^T of Q(sr + i si) (FP64 complex)
void launch_factor_complex(Problem& P, double sr, double si);
// complex FB solve in place on xn (N complex, interleaved, ND order); with vu
// the operator outputs of the complex shift: r_u = -Re x, r_l = Re(-s x) + v_u
void launch_fb_complex(Problem& P, void* xn, double sr, double si, const double* vu, double* ru,
                       double* rl);
// buffers and tensor-core plan of a precision, on first use (host work and
// allocations that rigaqep_factor keeps outside its timed region)
void prepare_factor(Problem& P, int precision);
// tensor-core products of the front factorisation (tcfront.cu)
void tc_plan(Problem& P, bool bf16);
void launch_tc_level(Problem& P, int level);
void tc_tuning_done(Problem& P);
bool tc_tuning_lookup(const Plan& L, bool bf16, std::vector<int32_t>& n35);
void tc_tuning_store(const Plan& L, bool bf16, const std::vector<int32_t>& n35);
void tc_plain_gemm(int m, int n, int K, const float* A, const float* B, float* C, bool bf16,
                   cudaStream_t s);
// relative residuals of FP64 refinement steps 1, 2, ... with the FP32 factor
std::vector<double> ir_history(Problem& P, double sigma, int max_steps, double target,
                               uint64_t seed);
void factor_configure(size_t smem_max);
void fb_plan(Problem& P);
void factor_plan(Problem& P);
// FB solve of Q x = b in the ND order, in place on xn (device, length N).
// If vu != nullptr the backward sweep writes r_u = -x to ru and
// r_l = sigma * r_u + vu to rl instead of writing x back (the operator step).
// With uscale != 1 (the scaled pencil) r_u = -uscale * x, r_l = -sigma x + vu.
void launch_fb(Problem& P, double* xn, double sigma, const double* vu, double* ru, double* rl,
               double uscale = 1.0);
void launch_gather(const int32_t* idx, const double* src, double* dst, int64_t n, int32_t ld_in,
                   int32_t ncol, cudaStream_t s);
void launch_scatter(const int32_t* idx, const double* src, double* dst, int64_t n, cudaStream_t s);
// the same for complex vectors (n pairs re, im)
void launch_gather2(const int32_t* idx, const double* src, double* dst, int64_t n, cudaStream_t s);
void launch_scatter2(const int32_t* idx, const double* src, double* dst, int64_t n, cudaStream_t s);
// Krylov pieces
void eigs_run(Problem& P, const EigsParams& E, const double* v1, double* lambda, double* X,
              double* eta, int* n_conv);
void grad_run(Problem& P, int neig, const double* lambda, const double* X, double* G);
void grad_run_noalloc(Problem& P, int neig, const double* lambda, const double* X, double* G);

}  // namespace rq

struct rigaqep_problem {
  rq::Problem impl;
};
