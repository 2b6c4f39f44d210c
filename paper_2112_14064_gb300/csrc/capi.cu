// C-ABI of rigaqep: argument checks, state machine and error mapping.
// Every entry point catches all C++ exceptions and returns a status code.
#include <algorithm>
#include <cmath>
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <utility>

#include "internal.h"

namespace rq {
namespace {
std::atomic<uint32_t> g_wait_limit{kDefaultWaitLimit};
}
uint32_t ritz_wait_limit() { return g_wait_limit.load(std::memory_order_relaxed); }
void set_ritz_wait_limit(uint32_t polls) {
  g_wait_limit.store(polls == 0 ? kDefaultWaitLimit : polls, std::memory_order_relaxed);
}
}  // namespace rq

namespace {

thread_local std::string g_last_error;

template <class F>
rigaqep_status guard(F&& f) {
  try {
    f();
    return RIGAQEP_OK;
  } catch (const rq::Error& e) {
    g_last_error = e.what();
    return e.code;
  } catch (const std::invalid_argument& e) {
    g_last_error = e.what();
    return RIGAQEP_ERR_ARG;
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return RIGAQEP_ERR_OOM;
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return RIGAQEP_ERR_INTERNAL;
  } catch (...) {
    g_last_error = "unknown failure";
    return RIGAQEP_ERR_INTERNAL;
  }
}

void need(bool cond, rigaqep_status code, const char* msg) {
  if (!cond) throw rq::Error(code, msg);
}

// complex-symmetric LDL^T of Q(sr + i si) into the handle's complex factor
void factor_complex(rq::Problem& P, double sr, double si) {
  P.factored = false;
  P.cand_valid = false;
  RQ_CUDA(cudaMemsetAsync(P.status.p, 0, sizeof(rq::DevStatus), P.stream));
  RQ_CUDA(cudaEventRecord(P.ev0, P.stream));
  rq::launch_factor_complex(P, sr, si);
  RQ_CUDA(cudaEventRecord(P.ev1, P.stream));
  rq::DevStatus st;
  RQ_CUDA(cudaMemcpyAsync(&st, P.status.p, sizeof(st), cudaMemcpyDeviceToHost, P.stream));
  RQ_CUDA(cudaStreamSynchronize(P.stream));
  float ms = 0.f;
  RQ_CUDA(cudaEventElapsedTime(&ms, P.ev0, P.ev1));
  P.info.factor_ms = ms;
  if (st.pivot_fail)
    throw rq::Error(RIGAQEP_ERR_PIVOT, "zero pivot in supernode " + std::to_string(st.pivot_fail - 1) +
                                           " of the complex factor");
  P.fact_fp32 = false;
  P.fact_prec = RIGAQEP_FP64;
  P.fact_gep = false;
  P.fact_cplx = true;
  P.fact_sigma = sr;
  P.fact_sigma_i = si;
  P.n_ir = 0;
  P.factored = true;
}

bool valid_precision(int32_t p) {
  return p == RIGAQEP_FP64 || p == RIGAQEP_TF32_IR || p == RIGAQEP_FP32_IR || p == RIGAQEP_BF16_IR;
}

void check_mesh(const rigaqep_mesh_desc* m) {
  need(m != nullptr, RIGAQEP_ERR_ARG, "mesh descriptor is NULL");
  need(m->ne_x == m->ne_y && m->ne_x >= 2, RIGAQEP_ERR_ARG, "only square meshes ne_x == ne_y >= 2");
  need(m->block_x == m->block_y, RIGAQEP_ERR_ARG, "block_x must equal block_y");
  need(m->p >= 2 && m->p <= rq::kMaxP, RIGAQEP_ERR_ARG, "p must be in [2, 8]");
  need(m->block_x >= 0 && (m->block_x == 0 || m->ne_x % m->block_x == 0), RIGAQEP_ERR_ARG,
       "block must be 0 or divide ne");
  need(m->n_quad >= 0 && m->n_quad <= 10, RIGAQEP_ERR_ARG, "n_quad must be in [0, 10]");
  need(m->leaf_min >= 0, RIGAQEP_ERR_ARG, "leaf_min must be >= 0");
}

template <class T, class A>
void copy_out(T* dst, const std::vector<T, A>& src) {
  if (dst && !src.empty()) std::memcpy(dst, src.data(), src.size() * sizeof(T));
}

}  // namespace

namespace rq {
cudaMemPool_t device_pool() {
  static std::mutex mu;
  static std::vector<cudaMemPool_t> pools;
  int dev = 0;
  RQ_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  if ((int)pools.size() <= dev) pools.resize(dev + 1, nullptr);
  if (!pools[dev]) {
    cudaMemPoolProps pp{};
    pp.allocType = cudaMemAllocationTypePinned;
    pp.handleTypes = cudaMemHandleTypeNone;
    pp.location.type = cudaMemLocationTypeDevice;
    pp.location.id = dev;
    cudaMemPool_t pool;
    RQ_CUDA(cudaMemPoolCreate(&pool, &pp));
    // keep up to 8 GiB cached between calls; more is returned at synchronisation
    uint64_t keep = 8ull << 30;
    RQ_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
    pools[dev] = pool;
  }
  return pools[dev];
}

void smem_at_least(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> cur;
  int dev = 0;
  RQ_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  size_t& c = cur[{dev, kernel}];
  if (bytes <= c) return;
  RQ_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  c = bytes;
}

Problem::~Problem() {
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
}
}  // namespace rq

struct rigaqep_symbolic {
  rq::Plan plan;
};

extern "C" {

rigaqep_status rigaqep_assemble(const rigaqep_mesh_desc* mesh, const double* sigma_e,
                                int32_t sigma_on_device, void* cuda_stream,
                                rigaqep_problem** out) {
  return guard([&] {
    need(out != nullptr, RIGAQEP_ERR_ARG, "out is NULL");
    *out = nullptr;
    check_mesh(mesh);
    need(sigma_e != nullptr, RIGAQEP_ERR_ARG, "sigma_e is NULL");
    rigaqep_problem* h = new rigaqep_problem();
    try {
      rq::Problem& P = h->impl;
      P.stream = (cudaStream_t)cuda_stream;
      rq::StreamScope scope(P.stream);
      RQ_CUDA(cudaGetDevice(&P.device));
      RQ_CUDA(cudaDeviceGetAttribute(&P.nsm, cudaDevAttrMultiProcessorCount, P.device));
      P.plan.build_pattern(mesh->ne_x, mesh->p, mesh->block_x, mesh->n_quad, mesh->leaf_min);
      RQ_CUDA(cudaEventCreate(&P.ev0));
      RQ_CUDA(cudaEventCreate(&P.ev1));
      P.rowptr.upload(P.plan.rowptr, P.stream);
      P.col.upload(P.plan.col, P.stream);
      int64_t ne2 = (int64_t)P.plan.ne * P.plan.ne;
      P.sigma_e.alloc(ne2);
      RQ_CUDA(cudaMemcpyAsync(P.sigma_e.p, sigma_e, sizeof(double) * ne2,
                              sigma_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                              P.stream));
      std::vector<double> hs(ne2);
      RQ_CUDA(cudaMemcpyAsync(hs.data(), P.sigma_e.p, sizeof(double) * ne2, cudaMemcpyDeviceToHost,
                              P.stream));
      RQ_CUDA(cudaStreamSynchronize(P.stream));
      P.sigma_min = *std::min_element(hs.begin(), hs.end());
      P.sigma_max = *std::max_element(hs.begin(), hs.end());
      P.status.alloc(1);
      RQ_CUDA(cudaMemsetAsync(P.status.p, 0, sizeof(rq::DevStatus), P.stream));
      rq::launch_assemble(P);
      rq::launch_norms(P);
      P.info.n1 = P.plan.n1;
      P.info.N = P.plan.N;
      P.info.nnz = P.plan.nnz;
    } catch (...) {
      delete h;
      throw;
    }
    *out = h;
  });
}

rigaqep_status rigaqep_analyze(rigaqep_problem* prob) {
  return guard([&] {
    need(prob != nullptr, RIGAQEP_ERR_ARG, "problem is NULL");
    rq::Problem& P = prob->impl;
    rq::StreamScope scope(P.stream);
    rq::Plan& L = P.plan;
    cudaStream_t s = P.stream;
    L.build_symbolic();
    P.perm.upload(L.perm, s);
    P.iperm.upload(L.iperm, s);
    P.sptr.upload(L.sptr, s);
    P.upd_ptr.upload(L.upd_ptr, s);
    P.upd_idx.upload(L.upd_idx, s);
    P.relmap.upload(L.relmap, s);
    P.child_ptr.upload(L.child_ptr, s);
    P.child_idx.upload(L.child_idx, s);
    P.lvl_nodes.upload(L.lvl_nodes, s);
    P.loff.upload(L.loff, s);
    P.uoff.upload(L.uoff, s);
    P.rowptr_n.upload(L.rowptr_n, s);
    rq::DBuf<int32_t> nd_err;
    nd_err.alloc(1);
    RQ_CUDA(cudaMemsetAsync(nd_err.p, 0, sizeof(int32_t), s));
    rq::launch_nd_csr(P, nd_err.p);
    rq::launch_permute_values(P);
    rq::launch_sell(P);
    P.lvl_maxF.assign(L.nlevels, 0);
    P.lvl_maxK.assign(L.nlevels, 0);
    for (int sn = 0; sn < L.nsuper; ++sn) {
      int k = L.sptr[sn + 1] - L.sptr[sn], u = L.upd_ptr[sn + 1] - L.upd_ptr[sn];
      int lv = L.level[sn];
      P.lvl_maxF[lv] = std::max(P.lvl_maxF[lv], k + u);
      P.lvl_maxK[lv] = std::max(P.lvl_maxK[lv], k);
    }
    P.Lval.alloc(L.l_total);
    P.Uval.alloc(L.u_total);
    P.Dinv.alloc(L.N);
    P.yvec.alloc(L.upd_idx.size());
    P.xwork.alloc(L.N);
    // fronts larger than the default 48 KB of dynamic shared memory
    size_t smax = sizeof(double) * (size_t)L.max_front;
    need(smax <= 200 * 1024, RIGAQEP_ERR_ARG, "front too large for one CTA");
    rq::factor_configure(smax);
    rq::fb_plan(P);
    rq::factor_plan(P);
    int32_t h_err = 0;
    RQ_CUDA(cudaMemcpyAsync(&h_err, nd_err.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    RQ_CUDA(cudaStreamSynchronize(s));
    need(h_err != 1, RIGAQEP_ERR_ARG, "a matrix row has more than 256 entries");
    if (h_err == 2) throw rq::Error(RIGAQEP_ERR_INTERNAL, "matrix entry outside the front");
    P.info.nsuper = L.nsuper;
    P.info.nlevels = L.nlevels;
    P.info.nnz_L = L.nnz_L;
    P.info.factor_flops = L.flops;
    P.info.max_front = L.max_front;
    P.analyzed = true;
    P.factored = false;
    P.cand_valid = false;
  });
}

rigaqep_status rigaqep_factor(rigaqep_problem* prob, double sigma, int32_t precision) {
  return guard([&] {
    need(prob != nullptr, RIGAQEP_ERR_ARG, "problem is NULL");
    rq::Problem& P = prob->impl;
    rq::StreamScope scope(P.stream);
    need(P.analyzed, RIGAQEP_ERR_STATE, "rigaqep_analyze must run before rigaqep_factor");
    need(valid_precision(precision), RIGAQEP_ERR_ARG,
         "precision must be RIGAQEP_FP64, RIGAQEP_TF32_IR, RIGAQEP_FP32_IR or RIGAQEP_BF16_IR");
    need(sigma == sigma, RIGAQEP_ERR_ARG, "sigma is NaN");
    const bool fp32 = precision != RIGAQEP_FP64;
    P.factored = false;
    P.cand_valid = false;
    RQ_CUDA(cudaMemsetAsync(P.status.p, 0, sizeof(rq::DevStatus), P.stream));
    rq::prepare_factor(P, precision);
    RQ_CUDA(cudaEventRecord(P.ev0, P.stream));
    rq::launch_factor(P, sigma, precision);
    RQ_CUDA(cudaEventRecord(P.ev1, P.stream));
    rq::DevStatus st;
    RQ_CUDA(cudaMemcpyAsync(&st, P.status.p, sizeof(st), cudaMemcpyDeviceToHost, P.stream));
    RQ_CUDA(cudaStreamSynchronize(P.stream));
    float ms = 0.f;
    RQ_CUDA(cudaEventElapsedTime(&ms, P.ev0, P.ev1));
    P.info.factor_ms = ms;
    if (st.timeout)
      throw rq::Error(RIGAQEP_ERR_TIMEOUT, "a bounded wait of the tensor-core front products ran out");
    if (st.pivot_fail)
      throw rq::Error(RIGAQEP_ERR_PIVOT, "non-positive pivot in supernode " +
                                             std::to_string(st.pivot_fail - 1) +
                                             ": Q(sigma) is not positive definite");
    P.fact_fp32 = fp32;
    P.fact_prec = precision;
    P.fact_gep = false;
    P.fact_cplx = false;
    P.info.tc_wide_levels = -1;
    if (precision == RIGAQEP_TF32_IR || precision == RIGAQEP_BF16_IR) {
      int64_t mask = 0;
      for (size_t l = 0; l < P.tc.n35.size() && l < 63; ++l)
        if (P.tc.n35[l] == 128) mask |= (int64_t)1 << l;
      P.info.tc_wide_levels = mask;
    }
    P.n_ir = 0;
    P.info.n_ir = 0;
    P.info.ir_residual = 0.0;
    if (fp32) {
      // refinement steps: the fewest that reach 1e-14 on a seeded right-hand
      // side, or the step after which the residual stops halving (at most 40)
      std::vector<double> h = rq::ir_history(P, sigma, 40, 1e-14, 0x5eedull);
      rq::DevStatus st2;
      RQ_CUDA(cudaMemcpyAsync(&st2, P.status.p, sizeof(st2), cudaMemcpyDeviceToHost, P.stream));
      RQ_CUDA(cudaStreamSynchronize(P.stream));
      if (st2.timeout)
        throw rq::Error(RIGAQEP_ERR_TIMEOUT, "a bounded wait between the FB work items ran out");
      int best = 0;
      double best_res = 1.0;
      for (size_t k = 0; k < h.size(); ++k)
        if (h[k] < best_res) {
          best_res = h[k];
          best = (int)k + 1;
        }
      if (best == 0 || !(best_res < 1e-6))
        throw rq::Error(RIGAQEP_ERR_REFINEMENT, "FP64 refinement with the low-precision factor "
                                                "does not contract (residual " + std::to_string(best_res) + ")");
      P.n_ir = best;
      P.info.n_ir = best;
      P.info.ir_residual = best_res;
    }
    P.factored = true;
    P.fact_sigma = sigma;
  });
}

rigaqep_status rigaqep_solve(rigaqep_problem* prob, const double* b, double* x, int32_t nrhs,
                             int32_t transpose) {
  return guard([&] {
    need(prob != nullptr, RIGAQEP_ERR_ARG, "problem is NULL");
    need(nrhs >= 0, RIGAQEP_ERR_ARG, "nrhs must be >= 0");
    need(nrhs == 0 || (b != nullptr && x != nullptr), RIGAQEP_ERR_ARG, "NULL argument");
    need(transpose == 0 || transpose == 1, RIGAQEP_ERR_ARG, "transpose must be 0 or 1");
    rq::Problem& P = prob->impl;
    rq::StreamScope scope(P.stream);
    need(P.factored, RIGAQEP_ERR_STATE, "rigaqep_factor must run before rigaqep_solve");
    need(!P.fact_cplx, RIGAQEP_ERR_STATE, "the factor is complex: use rigaqep_solve_complex");
    int64_t N = P.plan.N;
    // Q is symmetric, so the transposed solve uses the same factors and path.
    for (int c = 0; c < nrhs; ++c) {
      rq::launch_gather(P.perm.p, b + N * c, P.xwork.p, N, (int32_t)N, 1, P.stream);
      rq::launch_fb(P, P.xwork.p, P.fact_sigma, nullptr, nullptr, nullptr);
      rq::launch_scatter(P.perm.p, P.xwork.p, x + N * c, N, P.stream);
    }
    rq::DevStatus st;
    RQ_CUDA(cudaMemcpyAsync(&st, P.status.p, sizeof(st), cudaMemcpyDeviceToHost, P.stream));
    RQ_CUDA(cudaStreamSynchronize(P.stream));
    if (st.timeout)
      throw rq::Error(RIGAQEP_ERR_TIMEOUT, "a bounded wait between the FB work items ran out");
  });
}

rigaqep_status rigaqep_eigs(rigaqep_problem* prob, int32_t neig, double sigma,
                            const rigaqep_eigs_opts* opts, const double* v1, double* lambda,
                            double* X, double* eta, int32_t* n_converged) {
  rigaqep_status st = RIGAQEP_OK;
  rigaqep_status g = guard([&] {
    need(prob != nullptr && lambda != nullptr && X != nullptr && eta != nullptr &&
             n_converged != nullptr,
         RIGAQEP_ERR_ARG, "NULL argument");
    rq::Problem& P = prob->impl;
    rq::StreamScope scope(P.stream);
    need(P.analyzed, RIGAQEP_ERR_STATE, "rigaqep_analyze must run before rigaqep_eigs");
    rq::EigsParams E;
    E.neig = neig;
    E.target = sigma;
    E.in_region = opts && opts->shift_mode == RIGAQEP_SHIFT_IN_REGION;
    E.cplx = opts && opts->shift_mode == RIGAQEP_SHIFT_COMPLEX;
    need(!opts || opts->shift_mode == RIGAQEP_SHIFT_AT_TARGET || E.in_region || E.cplx,
         RIGAQEP_ERR_ARG, "unknown shift_mode");
    E.shift = (E.in_region || E.cplx) ? opts->shift : sigma;
    E.ncand = (E.in_region && opts->ncand > 0) ? opts->ncand : neig;
    if (E.cplx) {
      need(std::isfinite(opts->shift) && std::isfinite(opts->shift_imag) && opts->shift_imag > 0.0,
           RIGAQEP_ERR_ARG, "the complex shift needs a finite shift and shift_imag > 0");
      E.shift_i = opts->shift_imag;
      E.target = E.shift;
      E.ncand = opts->ncand > 0 ? opts->ncand : 2 * neig + 4;
      sigma = 1.0;   // the target argument is not used in this mode
    }
    E.m = opts && opts->krylov_dim > 0 ? opts->krylov_dim : std::min(rq::kMaxKrylov, 2 * E.ncand + 20);
    E.max_restarts = opts && opts->max_restarts > 0 ? opts->max_restarts : 1000;
    E.tol = opts && opts->tol > 0 ? opts->tol : 1e-10;
    E.seed = opts ? opts->seed : 1;
    need(!opts || opts->scaling == 0 || opts->scaling == 1, RIGAQEP_ERR_ARG, "scaling must be 0 or 1");
    E.vscale = (opts && opts->scaling == 1 && P.maxabs_M > 0.0) ? std::sqrt(P.maxabs_K / P.maxabs_M)
                                                                : 1.0;
    P.info.scale_factor = E.vscale;
    const int32_t prec = opts ? opts->precision : RIGAQEP_FP64;
    need(valid_precision(prec), RIGAQEP_ERR_ARG,
         "precision must be RIGAQEP_FP64, RIGAQEP_TF32_IR, RIGAQEP_FP32_IR or RIGAQEP_BF16_IR");
    need(neig >= 1 && neig <= E.ncand, RIGAQEP_ERR_ARG, "need 1 <= neig <= ncand");
    need(E.ncand < E.m && E.m <= rq::kMaxKrylov, RIGAQEP_ERR_ARG, "need ncand < krylov_dim <= 96");
    need(E.m <= 2 * P.plan.N, RIGAQEP_ERR_ARG, "krylov_dim exceeds 2N");
    need(sigma > 0.0, RIGAQEP_ERR_ARG, "the target must be real and positive");
    need(!E.in_region || E.shift == E.shift, RIGAQEP_ERR_ARG, "shift is NaN");
    need(!E.cplx || (prec == RIGAQEP_FP64 && !(opts && opts->scaling)), RIGAQEP_ERR_ARG,
         "the complex shift runs in FP64 without scaling");
    P.launches = 0;
    if (E.cplx) {
      if (!P.factored || !P.fact_cplx || P.fact_sigma != E.shift || P.fact_sigma_i != E.shift_i)
        factor_complex(P, E.shift, E.shift_i);
    } else if (!P.factored || P.fact_gep || P.fact_cplx || P.fact_sigma != E.shift ||
               P.fact_prec != prec) {
      rigaqep_status fs = rigaqep_factor(prob, E.shift, prec);
      if (fs != RIGAQEP_OK) throw rq::Error(fs, g_last_error);
    }
    int nconv = 0;
    rq::eigs_run(P, E, v1, lambda, X, eta, &nconv);
    *n_converged = nconv;
    if (nconv < neig) {
      g_last_error = "Krylov-Schur reached max_restarts before all wanted pairs converged";
      st = RIGAQEP_ERR_NO_CONVERGENCE;
    }
  });
  return g != RIGAQEP_OK ? g : st;
}

rigaqep_status rigaqep_grad_damping(rigaqep_problem* prob, int32_t neig, const double* lambda,
                                    const double* X, double* G) {
  return guard([&] {
    need(prob != nullptr && lambda != nullptr && X != nullptr && G != nullptr, RIGAQEP_ERR_ARG,
         "NULL argument");
    need(neig >= 1, RIGAQEP_ERR_ARG, "neig must be >= 1");
    rq::Problem& P = prob->impl;
    rq::StreamScope scope(P.stream);
    need(neig <= 64, RIGAQEP_ERR_ARG, "neig must be <= 64");
    rq::grad_run(P, neig, lambda, X, G);
  });
}

rigaqep_status rigaqep_grad_damping_noalloc(rigaqep_problem* prob, int32_t neig,
                                            const double* lambda, const double* X, double* G) {
  return guard([&] {
    need(prob != nullptr && lambda != nullptr && X != nullptr && G != nullptr, RIGAQEP_ERR_ARG,
         "NULL argument");
    // the scratch array is looked up for the current device and the kernels
    // run on the handle's stream: both must be the same GPU
    int dev = -1;
    RQ_CUDA(cudaGetDevice(&dev));
    need(dev == prob->impl.device, RIGAQEP_ERR_STATE,
         "the current device is not the device the problem was created on");
    rq::grad_run_noalloc(prob->impl, neig, lambda, X, G);
  });
}

rigaqep_status rigaqep_export_csr(const rigaqep_problem* prob, int32_t* rowptr, int32_t* col,
                                  double* K, double* M, double* C) {
  return guard([&] {
    need(prob != nullptr, RIGAQEP_ERR_ARG, "problem is NULL");
    const rq::Problem& P = prob->impl;
    rq::StreamScope scope(P.stream);
    copy_out(rowptr, P.plan.rowptr);
    copy_out(col, P.plan.col);
    size_t nb = sizeof(double) * P.plan.nnz;
    if (K) RQ_CUDA(cudaMemcpyAsync(K, P.K.p, nb, cudaMemcpyDeviceToHost, P.stream));
    if (M) RQ_CUDA(cudaMemcpyAsync(M, P.M.p, nb, cudaMemcpyDeviceToHost, P.stream));
    if (C) RQ_CUDA(cudaMemcpyAsync(C, P.C.p, nb, cudaMemcpyDeviceToHost, P.stream));
    RQ_CUDA(cudaStreamSynchronize(P.stream));
  });
}

rigaqep_status rigaqep_export_symbolic(const rigaqep_problem* prob, int32_t* perm, int32_t* sptr,
                                       int32_t* parent, int32_t* upd_ptr, int32_t* upd_idx,
                                       int32_t* level) {
  return guard([&] {
    need(prob != nullptr, RIGAQEP_ERR_ARG, "problem is NULL");
    const rq::Problem& P = prob->impl;
    rq::StreamScope scope(P.stream);
    need(P.analyzed, RIGAQEP_ERR_STATE, "rigaqep_analyze has not run");
    const rq::Plan& L = P.plan;
    copy_out(perm, L.perm);
    copy_out(sptr, L.sptr);
    copy_out(parent, L.parent);
    copy_out(upd_ptr, L.upd_ptr);
    copy_out(upd_idx, L.upd_idx);
    copy_out(level, L.level);
  });
}

rigaqep_status rigaqep_get_info(const rigaqep_problem* prob, rigaqep_info* info) {
  return guard([&] {
    need(prob != nullptr && info != nullptr, RIGAQEP_ERR_ARG, "NULL argument");
    rq::Problem& P = const_cast<rigaqep_problem*>(prob)->impl;
    if (P.analyzed) P.plan.exact_counts();   // once per handle, on the host
    *info = P.info;
    info->nnz_L_exact = P.analyzed ? P.plan.nnz_L_exact : -1;
    info->factor_flops_exact = P.analyzed ? P.plan.flops_exact : -1;
  });
}

rigaqep_status rigaqep_batch_eigs(rigaqep_problem* const* probs, int32_t nprob,
                                  rigaqep_batch_job* jobs, int32_t njobs, int32_t nthreads) {
  return guard([&] {
    need(probs != nullptr && nprob >= 1, RIGAQEP_ERR_ARG, "need at least one handle");
    need(njobs >= 0 && (njobs == 0 || jobs != nullptr), RIGAQEP_ERR_ARG, "jobs is NULL");
    need(nthreads >= 0, RIGAQEP_ERR_ARG, "nthreads must be >= 0");
    for (int32_t i = 0; i < nprob; ++i) {
      need(probs[i] != nullptr, RIGAQEP_ERR_ARG, "NULL handle in the batch");
      for (int32_t k = 0; k < i; ++k)
        need(probs[k] != probs[i], RIGAQEP_ERR_ARG, "a handle appears twice in the batch");
    }
    std::vector<std::vector<int32_t>> per(nprob);
    for (int32_t j = 0; j < njobs; ++j) {
      need(jobs[j].problem >= 0 && jobs[j].problem < nprob, RIGAQEP_ERR_ARG,
           "job refers to a handle outside the array");
      per[jobs[j].problem].push_back(j);
      jobs[j].status = RIGAQEP_ERR_STATE;   // overwritten when the job runs
      jobs[j].n_converged = jobs[j].certified = jobs[j].reused_candidates = 0;
      jobs[j].eigs_ms = 0.0;
    }
    // largest problems first (list scheduling of a ragged batch)
    std::vector<int32_t> order;
    for (int32_t i = 0; i < nprob; ++i)
      if (!per[i].empty()) order.push_back(i);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
      return probs[a]->impl.plan.N > probs[b]->impl.plan.N;
    });
    int dev = 0;
    RQ_CUDA(cudaGetDevice(&dev));
    std::vector<std::string> msg(njobs);
    std::atomic<int32_t> next{0};
    auto worker = [&]() {
      if (cudaSetDevice(dev) != cudaSuccess) return;   // jobs stay RIGAQEP_ERR_STATE
      for (;;) {
        int32_t q = next.fetch_add(1);
        if (q >= (int32_t)order.size()) return;
        rigaqep_problem* h = probs[order[q]];
        rigaqep_status st = RIGAQEP_OK;
        if (!h->impl.analyzed) st = rigaqep_analyze(h);
        for (int32_t j : per[order[q]]) {
          rigaqep_batch_job& J = jobs[j];
          rigaqep_status js = st;
          if (js == RIGAQEP_OK)
            js = rigaqep_eigs(h, J.neig, J.target, &J.opts, nullptr, J.lambda, J.X, J.eta,
                              &J.n_converged);
          J.status = js;
          if (js != RIGAQEP_OK) msg[j] = g_last_error;
          const rigaqep_info& inf = h->impl.info;
          J.certified = (int32_t)inf.certified;
          J.reused_candidates = (int32_t)inf.reused_candidates;
          J.eigs_ms = inf.eigs_ms;
        }
      }
    };
    int32_t nw = nthreads > 0 ? nthreads : 16;
    nw = std::max<int32_t>(1, std::min<int32_t>(nw, (int32_t)order.size()));
    std::vector<std::thread> th;
    for (int32_t t = 1; t < nw; ++t) th.emplace_back(worker);
    worker();
    for (auto& t : th) t.join();
    for (int32_t j = 0; j < njobs; ++j)
      if (jobs[j].status != RIGAQEP_OK)
        throw rq::Error((rigaqep_status)jobs[j].status,
                        "batch job " + std::to_string(j) + ": " +
                            (msg[j].empty() ? std::string("not run") : msg[j]));
  });
}

rigaqep_status rigaqep_symbolic_create(const rigaqep_mesh_desc* mesh, rigaqep_symbolic** out) {
  return guard([&] {
    need(out != nullptr, RIGAQEP_ERR_ARG, "out is NULL");
    *out = nullptr;
    check_mesh(mesh);
    rigaqep_symbolic* h = new rigaqep_symbolic();
    try {
      h->plan.build_pattern(mesh->ne_x, mesh->p, mesh->block_x, mesh->n_quad, mesh->leaf_min);
      h->plan.build_symbolic();
    } catch (...) {
      delete h;
      throw;
    }
    *out = h;
  });
}

rigaqep_status rigaqep_symbolic_counts(const rigaqep_symbolic* sym, int64_t* counts) {
  return guard([&] {
    need(sym != nullptr && counts != nullptr, RIGAQEP_ERR_ARG, "NULL argument");
    rq::Plan& L = const_cast<rigaqep_symbolic*>(sym)->plan;
    L.exact_counts();
    counts[0] = L.nnz_L;
    counts[1] = L.flops;
    counts[2] = L.nnz_L_exact;
    counts[3] = L.flops_exact;
  });
}

rigaqep_status rigaqep_symbolic_sizes(const rigaqep_symbolic* sym, int64_t* sizes) {
  return guard([&] {
    need(sym != nullptr && sizes != nullptr, RIGAQEP_ERR_ARG, "NULL argument");
    const rq::Plan& L = sym->plan;
    sizes[0] = L.N;
    sizes[1] = L.nnz;
    sizes[2] = L.nsuper;
    sizes[3] = (int64_t)L.upd_idx.size();
    sizes[4] = L.nlevels;
    sizes[5] = L.n1;
  });
}

rigaqep_status rigaqep_symbolic_export(const rigaqep_symbolic* sym, int32_t* perm, int32_t* sptr,
                                       int32_t* parent, int32_t* upd_ptr, int32_t* upd_idx,
                                       int32_t* level, int32_t* rowptr, int32_t* col) {
  return guard([&] {
    need(sym != nullptr, RIGAQEP_ERR_ARG, "NULL argument");
    const rq::Plan& L = sym->plan;
    copy_out(perm, L.perm);
    copy_out(sptr, L.sptr);
    copy_out(parent, L.parent);
    copy_out(upd_ptr, L.upd_ptr);
    copy_out(upd_idx, L.upd_idx);
    copy_out(level, L.level);
    copy_out(rowptr, L.rowptr);
    copy_out(col, L.col);
  });
}

void rigaqep_symbolic_destroy(rigaqep_symbolic* sym) { delete sym; }

const char* rigaqep_last_error(void) { return g_last_error.c_str(); }

void rigaqep_destroy(rigaqep_problem* prob) {
  if (!prob) return;
  if (prob->impl.stream) cudaStreamSynchronize(prob->impl.stream);
  delete prob;
}

}  // extern "C"

rigaqep_status rigaqep_front_gemm(int32_t precision, int32_t m, int32_t n, int32_t k,
                                  const float* A, const float* B, float* C, void* cuda_stream) {
  return guard([&] {
    need(precision == RIGAQEP_TF32_IR || precision == RIGAQEP_BF16_IR, RIGAQEP_ERR_ARG,
         "precision must be RIGAQEP_TF32_IR or RIGAQEP_BF16_IR");
    need(m >= 0 && n >= 0 && k >= 1, RIGAQEP_ERR_ARG, "need m, n >= 0 and k >= 1");
    need(m <= (1 << 20) && n <= (1 << 20) && k <= (1 << 16), RIGAQEP_ERR_ARG,
         "need m, n <= 2^20 and k <= 2^16");
    if (m == 0 || n == 0) return;
    need(A != nullptr && B != nullptr && C != nullptr, RIGAQEP_ERR_ARG, "NULL argument");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    rq::StreamScope scope(s);
    rq::tc_plain_gemm(m, n, k, A, B, C, precision == RIGAQEP_BF16_IR, s);
  });
}

void rigaqep_set_wait_limit(uint32_t polls) { rq::set_ritz_wait_limit(polls); }

namespace {

// LDL^T of K - mu M (FP64, pivots of either sign) into the handle's factor;
// returns the number of negative pivots
int64_t factor_gep(rq::Problem& P, double mu) {
  P.factored = false;
  P.cand_valid = false;
  RQ_CUDA(cudaMemsetAsync(P.status.p, 0, sizeof(rq::DevStatus), P.stream));
  RQ_CUDA(cudaEventRecord(P.ev0, P.stream));
  rq::launch_factor_gep(P, mu);
  RQ_CUDA(cudaEventRecord(P.ev1, P.stream));
  rq::DevStatus st;
  RQ_CUDA(cudaMemcpyAsync(&st, P.status.p, sizeof(st), cudaMemcpyDeviceToHost, P.stream));
  RQ_CUDA(cudaStreamSynchronize(P.stream));
  float ms = 0.f;
  RQ_CUDA(cudaEventElapsedTime(&ms, P.ev0, P.ev1));
  P.info.factor_ms = ms;
  if (st.pivot_fail)
    throw rq::Error(RIGAQEP_ERR_PIVOT, "zero pivot in supernode " + std::to_string(st.pivot_fail - 1) +
                                           ": mu is (numerically) an eigenvalue of a leading block");
  P.fact_fp32 = false;
  P.fact_prec = RIGAQEP_FP64;
  P.fact_gep = true;
  P.fact_cplx = false;
  P.fact_sigma = mu;
  P.n_ir = 0;
  P.factored = true;
  return st.neg_pivots;
}

}  // namespace

rigaqep_status rigaqep_inertia(rigaqep_problem* prob, double mu, int64_t* n_below) {
  return guard([&] {
    need(prob != nullptr && n_below != nullptr, RIGAQEP_ERR_ARG, "NULL argument");
    need(std::isfinite(mu), RIGAQEP_ERR_ARG, "mu must be finite");
    rq::Problem& P = prob->impl;
    rq::StreamScope scope(P.stream);
    need(P.analyzed, RIGAQEP_ERR_STATE, "rigaqep_analyze must run before rigaqep_inertia");
    *n_below = factor_gep(P, mu);
  });
}

rigaqep_status rigaqep_eigs_undamped(rigaqep_problem* prob, double mu_lo, double mu_hi,
                                     int32_t nmax, const rigaqep_eigs_opts* opts, const double* v1,
                                     double* mu, double* X, double* resid, int32_t* n_found,
                                     int32_t* count, int32_t* certified) {
  return guard([&] {
    need(prob != nullptr && n_found != nullptr && count != nullptr && certified != nullptr,
         RIGAQEP_ERR_ARG, "NULL argument");
    need(std::isfinite(mu_lo) && std::isfinite(mu_hi) && mu_lo < mu_hi, RIGAQEP_ERR_ARG,
         "need finite mu_lo < mu_hi");
    need(nmax >= 0, RIGAQEP_ERR_ARG, "nmax must be >= 0");
    need(!opts || opts->precision == RIGAQEP_FP64, RIGAQEP_ERR_ARG,
         "the undamped solve runs in FP64");
    rq::Problem& P = prob->impl;
    rq::StreamScope scope(P.stream);
    need(P.analyzed, RIGAQEP_ERR_STATE, "rigaqep_analyze must run before rigaqep_eigs_undamped");
    *n_found = 0;
    *certified = 0;
    P.launches = 0;
    // spectrum slicing: eigenvalues in [lo, hi) by Sylvester's law of inertia
    const int64_t below_lo = factor_gep(P, mu_lo);
    const int64_t below_hi = factor_gep(P, mu_hi);
    const int64_t cnt = below_hi - below_lo;
    need(cnt >= 0, RIGAQEP_ERR_INTERNAL, "inertia decreases with mu");
    *count = (int32_t)cnt;
    if (cnt == 0) {
      *certified = 1;
      return;
    }
    need(cnt <= nmax, RIGAQEP_ERR_ARG, "nmax is smaller than the number of eigenvalues in the interval");
    need(mu != nullptr && X != nullptr && resid != nullptr, RIGAQEP_ERR_ARG, "NULL output");
    rq::EigsParams E;
    E.gep = true;
    E.lo = mu_lo;
    E.hi = mu_hi;
    E.shift = 0.5 * (mu_lo + mu_hi);
    E.target = E.shift;
    E.in_region = false;
    const int extra = 4;
    E.m = opts && opts->krylov_dim > 0 ? opts->krylov_dim
                                       : std::min(rq::kMaxKrylov, 2 * (int)cnt + 2 * extra + 20);
    E.ncand = (int)cnt + extra;
    E.neig = (int)cnt;
    need(E.ncand < E.m && E.m <= rq::kMaxKrylov, RIGAQEP_ERR_ARG,
         "interval too wide for one slice: needs count + 4 < krylov_dim <= 96 (split it)");
    need(E.m <= P.plan.N, RIGAQEP_ERR_ARG, "krylov_dim exceeds N");
    E.max_restarts = opts && opts->max_restarts > 0 ? opts->max_restarts : 1000;
    E.tol = opts && opts->tol > 0 ? opts->tol : 1e-10;
    E.seed = opts ? opts->seed : 1;
    E.vscale = 1.0;
    factor_gep(P, E.shift);
    // start vector [0; v1] (v1: N entries, original order), or the upper
    // half dropped from the 2N seeded stream
    rq::DBuf<double> v2;
    if (v1) {
      v2.alloc(2 * P.plan.N);
      RQ_CUDA(cudaMemsetAsync(v2.p, 0, sizeof(double) * P.plan.N, P.stream));
      RQ_CUDA(cudaMemcpyAsync(v2.p + P.plan.N, v1, sizeof(double) * P.plan.N,
                              cudaMemcpyDeviceToDevice, P.stream));
    }
    rq::DBuf<double> lam, Xc;
    lam.alloc(2 * cnt);
    Xc.alloc(2 * (size_t)P.plan.N * cnt);
    int nconv = 0;
    rq::eigs_run(P, E, v1 ? v2.p : nullptr, lam.p, Xc.p, resid, &nconv);
    // n_found = converged candidates inside the interval
    const int nf = nconv;
    *n_found = nf;
    *certified = (nf == (int)cnt && P.gep_inside == (int)cnt && P.info.certified == 1) ? 1 : 0;
    P.info.certified = *certified;
    if (nf > 0) {
      // real parts: mu (lam holds (mu, 0)) and X (normalised real vectors)
      RQ_CUDA(cudaMemcpy2DAsync(mu, sizeof(double), lam.p, 2 * sizeof(double), sizeof(double), nf,
                                cudaMemcpyDeviceToDevice, P.stream));
      RQ_CUDA(cudaMemcpy2DAsync(X, sizeof(double), Xc.p, 2 * sizeof(double), sizeof(double),
                                (size_t)P.plan.N * nf, cudaMemcpyDeviceToDevice, P.stream));
    }
    RQ_CUDA(cudaStreamSynchronize(P.stream));
  });
}

rigaqep_status rigaqep_factor_complex(rigaqep_problem* prob, double sr, double si) {
  return guard([&] {
    need(prob != nullptr, RIGAQEP_ERR_ARG, "problem is NULL");
    need(std::isfinite(sr) && std::isfinite(si), RIGAQEP_ERR_ARG, "the shift must be finite");
    rq::Problem& P = prob->impl;
    rq::StreamScope scope(P.stream);
    need(P.analyzed, RIGAQEP_ERR_STATE, "rigaqep_analyze must run before rigaqep_factor_complex");
    factor_complex(P, sr, si);
  });
}

rigaqep_status rigaqep_solve_complex(rigaqep_problem* prob, const double* b, double* x,
                                     int32_t nrhs) {
  return guard([&] {
    need(prob != nullptr, RIGAQEP_ERR_ARG, "problem is NULL");
    need(nrhs >= 0, RIGAQEP_ERR_ARG, "nrhs must be >= 0");
    need(nrhs == 0 || (b != nullptr && x != nullptr), RIGAQEP_ERR_ARG, "NULL argument");
    rq::Problem& P = prob->impl;
    rq::StreamScope scope(P.stream);
    need(P.factored && P.fact_cplx, RIGAQEP_ERR_STATE,
         "rigaqep_factor_complex must run before rigaqep_solve_complex");
    const int64_t N = P.plan.N;
    for (int c = 0; c < nrhs; ++c) {
      // gather/scatter the (re, im) pairs as 16-byte elements in the ND order
      rq::launch_gather2(P.perm.p, b + 2 * N * c, (double*)P.cx.y.p, N, P.stream);
      rq::launch_fb_complex(P, P.cx.y.p, P.fact_sigma, P.fact_sigma_i, nullptr, nullptr, nullptr);
      rq::launch_scatter2(P.perm.p, (const double*)P.cx.y.p, x + 2 * N * c, N, P.stream);
    }
    rq::DevStatus st;
    RQ_CUDA(cudaMemcpyAsync(&st, P.status.p, sizeof(st), cudaMemcpyDeviceToHost, P.stream));
    RQ_CUDA(cudaStreamSynchronize(P.stream));
    if (st.timeout)
      throw rq::Error(RIGAQEP_ERR_TIMEOUT, "a bounded wait between the FB work items ran out");
  });
}
