/*
 * rigaqep — shift-and-invert solver for quadratic eigenvalue problems from
 * refined isogeometric (rIGA) discretisations, on one GB300 GPU (sm_103a).
 *
 * Problem (paper, Eq. QuadEig, Section 4.2):  (K + lambda C + lambda^2 M) u = 0
 * with K the Laplacian stiffness, M the mass matrix and C = sum_e sigma_e M_e
 * (per-element damping) of degree-p tensor-product B-splines on the unit
 * square, homogeneous Dirichlet boundary.  rIGA repeats the knots on every
 * block-th element line p times (C^0 separators, Section 3.3); block = 0 is
 * maximum-continuity IGA (Section 3.2).
 *
 * Pipeline, in call order (Algorithm 2 of the paper):
 *   rigaqep_assemble  Gauss-quadrature K, M, C in CSR           (Section 3)
 *   rigaqep_analyze   separator nested dissection + symbolic    (Section 3.3)
 *   rigaqep_factor    multifrontal LDL^T of Q(s)=s^2M+sC+K      (Alg. 2, "Factorize Q(s)")
 *   rigaqep_solve     forward/backward substitution with the factors (Section 4.2.2)
 *   rigaqep_eigs      Krylov-Schur on the linearised pencil     (Eqs. Linearization,
 *                     BlockOperatorVector; Algorithms 1 and 2; Section 4.1.3)
 *   rigaqep_grad_damping  d lambda / d sigma_e                   (no counterpart in the paper)
 *
 * Conventions for every entry point:
 *  - Return value: RIGAQEP_OK or an error code; nothing is thrown across the
 *    ABI and the process is never terminated.  rigaqep_last_error() gives a
 *    message for the calling thread's last failure.
 *  - DOF numbering: dof = i + n*j (xi index i fastest), n DOFs per direction
 *    after removing the Dirichlet functions.  Element numbering e = ex + ne*ey.
 *  - Pointers marked "device" must be CUDA device memory of the current
 *    device; "host" pointers are ordinary host memory.  Caller buffers are
 *    borrowed for the duration of the call only.  All device work runs on the
 *    stream given to rigaqep_assemble; calls that return host values
 *    synchronise that stream.
 *  - The handle owns every internal device buffer (CSR, factors, Krylov
 *    basis) and frees them in rigaqep_destroy.
 *  - Out-of-order calls (e.g. solve before factor) return RIGAQEP_ERR_STATE.
 */
#ifndef RIGAQEP_H
#define RIGAQEP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rigaqep_problem rigaqep_problem;
typedef struct rigaqep_symbolic rigaqep_symbolic;

typedef enum {
  RIGAQEP_OK = 0,
  RIGAQEP_ERR_ARG = 1,             /* invalid argument (sizes, NULL, ranges) */
  RIGAQEP_ERR_STATE = 2,           /* call out of order */
  RIGAQEP_ERR_CUDA = 3,            /* a CUDA runtime call failed */
  RIGAQEP_ERR_OOM = 4,             /* device or host allocation failed */
  RIGAQEP_ERR_PIVOT = 5,           /* non-positive pivot in LDL^T (Q(s) not SPD) */
  RIGAQEP_ERR_REFINEMENT = 6,      /* iterative refinement of the low-precision factor
                                      does not contract (rigaqep_factor) */
  RIGAQEP_ERR_NO_CONVERGENCE = 7,  /* max_restarts reached; partial results returned */
  RIGAQEP_ERR_TIMEOUT = 8,         /* a bounded device-side wait gave up */
  RIGAQEP_ERR_INTERNAL = 9         /* a device-side consistency check failed */
} rigaqep_status;

/* Mesh and discretisation.  ne_x = ne_y = ne (square meshes only), p >= 2,
 * block = 0 (IGA) or a divisor of ne (rIGA C^0 lines every block elements),
 * n_quad = Gauss points per direction (0 selects p+1, exact for M_e, K_e),
 * leaf_min = largest box extent left undissected inside a macroelement
 * (0 selects 8). */
typedef struct {
  int32_t ne_x, ne_y, p, block_x, block_y, n_quad, leaf_min;
} rigaqep_mesh_desc;

/* Factor precision (the paper does not state its own; these are the
 * mixed-precision forms of Algorithm 2's "Factorize Q(s)" and of the solves of
 * Section 4.2.2).
 *  RIGAQEP_FP64: FP64 fronts and solves.
 *  RIGAQEP_FP32_IR: FP32 fronts (SIMT) and FP32 forward/backward sweeps,
 *    every solve refined in FP64 (x += Q32^{-1}(y - Q x) with the FP64
 *    residual of the assembled K, M, C) for a number of steps chosen when
 *    the factor is made (info.n_ir).
 *  RIGAQEP_TF32_IR: as FP32_IR, with the dense products of every front
 *    (L21 = F21 inv(L11)^T D^{-1}, the Schur update U -= L21 D L21^T and
 *    W = L21 inv(L11)) on the tensor cores in TF32 with FP32 accumulation;
 *    each operand is split into two TF32 terms (hi + lo, 22 significant bits)
 *    and the product is hi*hi + hi*lo + lo*hi.  Pivot blocks stay FP32.
 *  RIGAQEP_BF16_IR: the same products in BF16 (two BF16 terms, 16 bits),
 *    with the pivot-scaled operands of each front multiplied by a power of
 *    two that brings them near 1. */
typedef enum {
  RIGAQEP_FP64 = 0,
  RIGAQEP_TF32_IR = 1,
  RIGAQEP_FP32_IR = 2,
  RIGAQEP_BF16_IR = 3
} rigaqep_precision;

/* Krylov-Schur options.  krylov_dim = m (neig < m <= 96), max_restarts
 * (0 selects 1000), tol = Ritz-estimate tolerance |h_{m+1,m} y_m|/|theta|
 * (0 selects 1e-10), seed = start-vector seed used when no start vector is
 * given (v1[i] = splitmix64(seed+i)/2^64 - 0.5 over the 2N entries).
 *
 * shift_mode selects where the spectral transformation is placed:
 *  RIGAQEP_SHIFT_AT_TARGET (0): the shift is the target sigma itself, as in
 *    the paper (Section 4.1.1, Algorithm 2); the neig Ritz pairs nearest
 *    sigma are converged and returned.
 *  RIGAQEP_SHIFT_IN_REGION (1): Q(shift) is factorised at opts->shift (a real
 *    shift inside the spectrum region; Q(shift) must be SPD, shift = 0 gives
 *    Q = K), the ncand pairs nearest the shift are converged, and the neig of
 *    them nearest the target sigma are returned.  The selection is certified
 *    (info.certified = 1) when no other eigenvalue can be nearer the target,
 *    assuming that every eigenvalue not converged lies at least r from the
 *    shift (r = the largest candidate distance; Krylov-Schur converges the
 *    eigenvalues nearest the shift first, but the call does not prove that
 *    none was skipped), since complex eigenvalues have
 *    Re lambda in [-max sigma_e / 2, -min sigma_e / 2] (Rayleigh quotients of
 *    the QEP with K, M SPD and C = sum sigma_e M_e, sigma_e >= 0) and real
 *    ones are <= 0, which bounds their distance to the target from below. */
enum { RIGAQEP_SHIFT_AT_TARGET = 0, RIGAQEP_SHIFT_IN_REGION = 1, RIGAQEP_SHIFT_COMPLEX = 2 };
/* RIGAQEP_SHIFT_COMPLEX (2): the shift is the complex number s = opts->shift +
 *    i opts->shift_imag (shift_imag > 0; Section 4.1.1 allows s in C; with
 *    s = i sqrt(sigma) the eigenvalues nearest s are the modes of angular
 *    frequency near sqrt(sigma)).  Q(s) is factorised as a complex symmetric
 *    LDL^T (FP64), and the Krylov iteration runs on the real operator
 *    Re((A - s B)^{-1} B), whose eigenvalue for an eigenvalue lambda of the
 *    pencil is (1/(lambda - s) + 1/(lambda - conj s)) / 2; each converged one
 *    gives two roots of a quadratic, and the eigenvector decides between them
 *    (the smaller backward error).  The neig eigenvalues nearest s among the
 *    ncand converged candidates (0 selects 2 neig + 4: the iteration also
 *    converges the conjugates near conj s) are returned, nearest first; the
 *    `sigma` argument of rigaqep_eigs is not used, and info.certified is 0
 *    (no distance certificate).  FP64 only. */
typedef struct {
  int32_t krylov_dim;
  int32_t max_restarts;
  double tol;
  uint64_t seed;
  int32_t precision;
  int32_t shift_mode;
  double shift;
  int32_t ncand;         /* pairs converged around the shift (0 selects neig) */
  int32_t scaling;       /* 1: solve the scaled pencil of Remark 4 (below); 0: unscaled */
  double shift_imag;     /* imaginary part of the shift (RIGAQEP_SHIFT_COMPLEX) */
} rigaqep_eigs_opts;
/* Scaling (paper, Remark 4): with varsigma = sqrt(max|K_ij| / max|M_ij|)
 * (the "infinity norm" of the paper is the largest absolute entry), the
 * Krylov iteration runs on K + gamma C_s + gamma^2 M_s with C_s = varsigma C,
 * M_s = varsigma^2 M and gamma = lambda / varsigma: the same shifted factor
 * Q(s), the operator and B-inner product of the scaled linearisation, and
 * lambda = varsigma gamma on output (info.scale_factor = varsigma).  In exact
 * arithmetic the eigenpairs are those of the unscaled call. */

/* Sizes and counters of a handle (host struct filled by rigaqep_get_info). */
typedef struct {
  int64_t n1;            /* DOFs per direction */
  int64_t N;             /* total DOFs */
  int64_t nnz;           /* entries of the shared K/M/C pattern */
  int64_t nsuper;        /* supernodes (= fronts) */
  int64_t nlevels;       /* assembly-tree levels */
  int64_t nnz_L;         /* supernodal factor entries, dense pivot blocks (stored and read) */
  int64_t factor_flops;  /* sum_j (c_j^2 + 2 c_j), c_j = off-diagonals of column j in the
                            supernodal structure (the arithmetic the fronts execute) */
  int64_t max_front;     /* largest front order k+u */
  int64_t n_apply;       /* operator applications (FB solves) of the last eigs */
  int64_t n_restarts;    /* Krylov-Schur restarts of the last eigs */
  int64_t n_spmv;        /* sparse matrix-vector products of the last eigs */
  int64_t n_vv;          /* length-N vector-vector products of the last eigs */
  int64_t n_qr_sweeps;   /* Francis QR sweeps of the Ritz steps of the last eigs */
  double norm_K, norm_M, norm_C;  /* max-row-sum norms */
  double factor_ms;      /* device time of the last rigaqep_factor */
  double eigs_ms;        /* device time of the last rigaqep_eigs */
  double fb_ms;          /* device time of its FB solves: CUDA events around every
                            eighth solve, their mean times n_apply */
  int64_t certified;     /* 1: no eigenvalue outside the converged candidates can be nearer
                            the target than the returned pairs, given that the candidates
                            include every eigenvalue within their largest distance to the
                            shift (what Krylov-Schur converges first, not proved by the
                            call; checked against dense eigensolves in the tests) */
  double cert_margin;    /* lower bound on the distance of any other eigenvalue to the
                            target, minus the largest returned distance (>= 0 when certified) */
  int64_t n_launches;    /* kernels launched by the last eigs (including its factorisation) */
  double ritz_ms;        /* device time of its Ritz/restart steps */
  double ritz_phase_cycles[6];  /* SM cycles of those steps by phase: Hessenberg reduction,
                                   QR sweeps, eigenvalues and ranks, Ritz vectors and
                                   estimates, reordering, locking */
  int64_t n_ir;           /* FP64 refinement steps per solve (0 with the FP64 factor) */
  double ir_residual;     /* relative residual reached by those steps on the probe */
  int64_t reused_candidates;  /* 1: the last eigs reused the converged candidates of the
                                 previous in-region call (same factor, shift, ncand,
                                 krylov_dim, tol, max_restarts, seed; seeded start) and
                                 only selected and extracted for its target */
  int64_t nnz_L_exact;        /* structurally non-zero entries of L (diagonal included)
                                 with the exact column counts: the algorithmic factor
                                 size (-1 before rigaqep_analyze) */
  int64_t factor_flops_exact; /* sum_j (c_j^2 + 2 c_j) with the exact column counts: the
                                 algorithmic factorisation flops (-1 before analyze) */
  double scale_factor;        /* varsigma of the last eigs (1 when it was not scaled) */
  int64_t tc_wide_levels;     /* TF32/BF16 factor: bit l set when tree level l computes its
                                 L21 product in 128-column tiles (else 64), as chosen by the
                                 library's autotuner (both timed on the first tensor-core
                                 factorisation of the mesh in the process); -1 otherwise */
} rigaqep_info;

/* Create a handle and assemble K, M, C (original DOF order, one CSR
 * pattern, FP64).  sigma_e: ne*ne coefficients, element ex + ne*ey, host
 * memory if sigma_on_device == 0, else device memory.  cuda_stream: a
 * cudaStream_t (NULL = legacy default stream).  On success *out owns all
 * device memory of the problem; on failure *out is NULL.
 * Defined by: Section 3.1 (tensor-product B-splines, Cox-de Boor), Section
 * 3.3 (rIGA knots), Section 2 forms a, b, c in their scalar H^1 analogue. */
rigaqep_status rigaqep_assemble(const rigaqep_mesh_desc* mesh, const double* sigma_e,
                                int32_t sigma_on_device, void* cuda_stream,
                                rigaqep_problem** out);

/* Integer symbolic phase: canonical separator nested dissection, supernodes,
 * assembly tree, update structures, extend-add maps and level sets, then the
 * ND-ordered device CSR.  Bit-exact and deterministic.
 * Defined by: Section 3.3 (separators coincide with the solver's partitions)
 * and Section 5.1 (multifrontal solver with nested-dissection ordering). */
rigaqep_status rigaqep_analyze(rigaqep_problem* prob);

/* Numeric multifrontal LDL^T of Q(sigma) = sigma^2 M + sigma C + K, fronts
 * batched per tree level, in the given rigaqep_precision.  Requires analyze.
 * A non-positive pivot returns RIGAQEP_ERR_PIVOT (Q(sigma) is SPD for real
 * sigma > 0).  With RIGAQEP_FP32_IR the call also chooses the number of FP64
 * refinement steps per solve: the smallest count (at most 40) after which a
 * seeded right-hand side reaches a relative residual of 1e-14 or stops
 * improving; RIGAQEP_ERR_REFINEMENT if the refinement does not contract.
 * Defined by: Algorithm 2 ("Factorize Q(s)"), Section 4.2.1. */
rigaqep_status rigaqep_factor(rigaqep_problem* prob, double sigma, int32_t precision);

/* Complex-symmetric LDL^T of Q(s) = s^2 M + s C + K at s = sr + i si (FP64
 * complex, no pivoting; every leading block of Q(s) is non-singular when
 * si != 0 and all sigma_e > 0, its imaginary part si (C + 2 sr M) being
 * definite for sr >= 0), replacing the handle's factor; then
 * rigaqep_solve_complex.  RIGAQEP_ERR_PIVOT on a zero pivot.
 * Defined by: Algorithm 2 ("Factorize Q(s)") with s in C (Section 4.1.1). */
rigaqep_status rigaqep_factor_complex(rigaqep_problem* prob, double sr, double si);

/* x = Q(s)^{-1} b with the complex factor: b, x device arrays of N complex
 * values (interleaved re, im; original DOF order), nrhs right-hand sides
 * (column-major N x nrhs complex); b and x may alias.
 * Defined by: Section 4.2.2 (forward/backward elimination). */
rigaqep_status rigaqep_solve_complex(rigaqep_problem* prob, const double* b, double* x,
                                     int32_t nrhs);

/* x = Q(sigma)^{-1} b for nrhs right-hand sides (device, original DOF order,
 * column-major N x nrhs; b and x may alias; both may be NULL when nrhs = 0).
 * transpose = 1 solves with Q^T, which equals Q (K, M, C symmetric): the
 * same factors and path.
 * Defined by: Section 4.2.2 (forward/backward elimination). */
rigaqep_status rigaqep_solve(rigaqep_problem* prob, const double* b, double* x,
                             int32_t nrhs, int32_t transpose);

/* neig eigenpairs of the QEP nearest the real target sigma by shift-and-invert
 * Krylov-Schur on the linearised 2N pencil (factors Q at the shift chosen by
 * opts->shift_mode if it is not factorised there already).
 * v1: optional device start vector of 2N entries (original order; NULL =
 * splitmix64 from opts->seed).  Outputs (device): lambda 2*neig doubles
 * (re, im) ordered by |lambda - sigma| with Im > 0 first on ties; X N*neig
 * complex (interleaved re, im; column k = eigenvector k, original order, unit
 * 2-norm, largest-modulus entry real positive); eta neig backward errors
 * ||Q(lambda)x|| / ((|lambda|^2||M|| + |lambda|||C|| + ||K||)||x||).
 * *n_converged (host) = wanted pairs whose Ritz estimate met tol.
 * Returns RIGAQEP_ERR_NO_CONVERGENCE (with outputs filled) if max_restarts
 * is reached first.
 * Defined by: Eqs. (Linearization), (BlockOperatorVector), Algorithm 1
 * (Arnoldi, B-inner product), Algorithm 2, Eq. (ArnoldiRitz), Section 4.1.3. */
rigaqep_status rigaqep_eigs(rigaqep_problem* prob, int32_t neig, double sigma,
                            const rigaqep_eigs_opts* opts, const double* v1,
                            double* lambda, double* X, double* eta,
                            int32_t* n_converged);
/* In-region calls (shift_mode RIGAQEP_SHIFT_IN_REGION, v1 == NULL) that
 * repeat the previous call's shift, ncand, krylov_dim, tol, max_restarts and
 * seed on the same factor reuse its converged candidates and only select and
 * extract the pairs for the new target and neig (info.reused_candidates = 1):
 * the Krylov iteration does not depend on the target in that mode, so the
 * result is the one a fresh call would return. */

/* One eigensolve of a batch (rigaqep_batch_eigs).  Inputs: problem (index
 * into the handle array), neig, target, opts (as for rigaqep_eigs; the start
 * vector is always the seeded one), lambda/X/eta (device outputs laid out as
 * for rigaqep_eigs, owned by the caller).  Outputs: n_converged, status (the
 * rigaqep_status of this job), certified and reused_candidates (as in
 * rigaqep_info after the job) and eigs_ms (its device time). */
typedef struct {
  int32_t problem;
  int32_t neig;
  double target;
  rigaqep_eigs_opts opts;
  double* lambda;
  double* X;
  double* eta;
  int32_t n_converged;
  int32_t status;
  int32_t certified;
  int32_t reused_candidates;
  double eigs_ms;
} rigaqep_batch_job;

/* Many eigensolves of many independent QEPs (problems of uneven size, several
 * targets each) in one call.  Every handle must be assembled on the calling
 * thread's current device; handles not yet analysed are analysed here.  The
 * jobs of one handle run in the order given, on that handle's stream, on one
 * host worker thread; different handles run concurrently on up to nthreads
 * workers (0 = one per handle, at most 16), largest N first.  Handles
 * created on distinct streams overlap on the GPU; handles sharing a stream
 * are correct but serialised.  Jobs with consecutive in-region solves of one
 * handle share its Krylov iteration (see rigaqep_eigs).  A handle may appear
 * in the array only once.  Returns RIGAQEP_OK when every job returned
 * RIGAQEP_OK, else the status of the lowest-indexed failing job (its message
 * in rigaqep_last_error); every job's own status is always written.  The call
 * returns after all jobs have completed on the device.
 * Defined by: no counterpart in the paper (which solves one problem at a
 * time); each job is the solve of rigaqep_eigs. */
rigaqep_status rigaqep_batch_eigs(rigaqep_problem* const* probs, int32_t nprob,
                                  rigaqep_batch_job* jobs, int32_t njobs, int32_t nthreads);

/* G[k, e] = d lambda_k / d sigma_e = -lambda_k x_e^T M_e x_e / x^T(2 lambda_k M + C) x
 * (unconjugated: the left eigenvector of the symmetric QEP is x itself).
 * lambda (2*neig) and X (N*neig complex) as returned by rigaqep_eigs (device);
 * G: device, neig x ne^2 complex, row-major (re, im interleaved).
 * The paper has no sensitivity analysis; this is first-order perturbation
 * theory of a simple eigenvalue of Eq. (QuadEig). */
rigaqep_status rigaqep_grad_damping(rigaqep_problem* prob, int32_t neig,
                                    const double* lambda, const double* X, double* G);

/* The same d lambda / d sigma_e as rigaqep_grad_damping (same arguments and
 * layout), for callers that must not allocate device memory during the call:
 * code that runs on a latency-critical path where the implicit device-wide
 * synchronisation of cudaMalloc/cudaFree would stall other streams, or code
 * inside a framework whose memory manager owns all device memory.  The
 * paper has no counterpart; this is a service of the library.
 * Its reduction scratch is a fixed array in device global memory (305 KiB,
 * held by every GPU that loads the library until the process exits), so
 * neig must be <= 64; larger neig returns RIGAQEP_ERR_ARG before any GPU
 * work.  The first call on each device looks up that array's device address
 * with the device current; make that first call before any stream capture.
 * All calls share the one array (each call writes every entry it reads), so
 * calls that overlap on the GPU, from any stream or thread, race: serialise
 * them.  Synchronises the handle's stream before returning. */
rigaqep_status rigaqep_grad_damping_noalloc(rigaqep_problem* prob, int32_t neig,
                                            const double* lambda, const double* X, double* G);

/* The dense product of the front factorisation's tensor-core path, on its
 * own: C = A B^T with A (m x k), B (n x k) and C (m x n) row-major FP32
 * device arrays, computed by the same operand staging (two-term split) and
 * tcgen05 kernels as the RIGAQEP_TF32_IR / RIGAQEP_BF16_IR fronts, on
 * cuda_stream (a cudaStream_t; NULL = legacy default).  m, n <= 2^20,
 * k <= 2^16; m = 0 or n = 0 does nothing.  Allocates its staging buffers
 * from the library's pool; synchronises the stream.  Returns
 * RIGAQEP_ERR_TIMEOUT if a bounded wait of the pipeline ran out.
 * Defined by: Algorithm 2 ("Factorize Q(s)"): the Schur-complement and panel
 * products of each front are this product. */
rigaqep_status rigaqep_front_gemm(int32_t precision, int32_t m, int32_t n, int32_t k,
                                  const float* A, const float* B, float* C, void* cuda_stream);

/* Undamped pencil K x = mu M x (the QEP without its damping term, lambda =
 * +-i sqrt(mu)): the number of its eigenvalues mu' < mu, by Sylvester's law
 * of inertia from the negative pivots of the LDL^T of K - mu M (spectrum
 * slicing, Section 4.1.4).  The factorisation (FP64, pivots of either sign,
 * no pivoting) replaces the handle's factor.  *n_below: host.  Returns
 * RIGAQEP_ERR_PIVOT if a pivot is zero (mu is, in floating point, an
 * eigenvalue of a leading block of the nested-dissection order).
 * Defined by: Section 4.1.4 (spectrum slicing). */
rigaqep_status rigaqep_inertia(rigaqep_problem* prob, double mu, int64_t* n_below);

/* Every eigenpair of the undamped pencil K x = mu M x with mu in [mu_lo,
 * mu_hi): *count (host) = inertia(mu_hi) - inertia(mu_lo) eigenvalues lie
 * there; shift-and-invert Lanczos at the midpoint (operator (K - s M)^{-1} M
 * in the M-inner product, full reorthogonalisation, thick restarts of the
 * Krylov-Schur kind; Remark 3) converges count + 4 pairs nearest it and
 * returns those inside the interval, ascending.  Outputs (device): mu
 * (count values), X (N x count real, column-major, original order, unit
 * 2-norm, largest entry positive), resid (count backward errors
 * ||K x - mu M x|| / ((||K|| + |mu| ||M||) ||x||)); *n_found (host)
 * converged pairs inside; *certified (host) = 1 when exactly *count
 * converged pairs were found inside.  nmax bounds the outputs
 * (RIGAQEP_ERR_ARG with *count set if count > nmax); count + 4 must be below
 * the Krylov dimension (<= 96): split wider intervals.  opts: krylov_dim,
 * max_restarts, tol, seed as for rigaqep_eigs (precision FP64 only; the
 * other fields are ignored); v1: optional device start vector of N entries
 * (NULL: entries N..2N-1 of the seeded 2N stream).  Three factorisations
 * (lo, hi, midpoint) replace the handle's factor.
 * Defined by: Remark 3 (Lanczos), Section 4.1.4 (spectrum slicing). */
rigaqep_status rigaqep_eigs_undamped(rigaqep_problem* prob, double mu_lo, double mu_hi,
                                     int32_t nmax, const rigaqep_eigs_opts* opts, const double* v1,
                                     double* mu, double* X, double* resid, int32_t* n_found,
                                     int32_t* count, int32_t* certified);

/* Copy the original-order CSR (rowptr N+1, col nnz int32; K, M, C nnz
 * doubles) to host buffers; any pointer may be NULL to skip it. */
rigaqep_status rigaqep_export_csr(const rigaqep_problem* prob, int32_t* rowptr, int32_t* col,
                                  double* K, double* M, double* C);

/* Copy the symbolic phase to host buffers (any may be NULL): perm[N]
 * (perm[new] = old dof), sptr[nsuper+1], parent[nsuper] (-1 = root),
 * upd_ptr[nsuper+1], upd_idx[upd_ptr[nsuper]] (new indices, ascending),
 * level[nsuper]. */
rigaqep_status rigaqep_export_symbolic(const rigaqep_problem* prob, int32_t* perm, int32_t* sptr,
                                       int32_t* parent, int32_t* upd_ptr, int32_t* upd_idx,
                                       int32_t* level);

/* Sizes and counters (host struct). */
rigaqep_status rigaqep_get_info(const rigaqep_problem* prob, rigaqep_info* info);

/* Host-only planning (no CUDA call, usable without a GPU): the same CSR
 * pattern and symbolic phase as assemble + analyze.  sizes[0..5] =
 * {N, nnz, nsuper, n_upd, nlevels, n1}. */
rigaqep_status rigaqep_symbolic_create(const rigaqep_mesh_desc* mesh, rigaqep_symbolic** out);
rigaqep_status rigaqep_symbolic_sizes(const rigaqep_symbolic* sym, int64_t* sizes);
rigaqep_status rigaqep_symbolic_export(const rigaqep_symbolic* sym, int32_t* perm, int32_t* sptr,
                                       int32_t* parent, int32_t* upd_ptr, int32_t* upd_idx,
                                       int32_t* level, int32_t* rowptr, int32_t* col);
/* counts[0..3] = {nnz_L, factor_flops, nnz_L_exact, factor_flops_exact} of the
 * plan, with the meaning of the rigaqep_info fields of those names; host only. */
rigaqep_status rigaqep_symbolic_counts(const rigaqep_symbolic* sym, int64_t* counts);
void rigaqep_symbolic_destroy(rigaqep_symbolic* sym);

/* Number of polls after which a wait between the cooperating CTAs of the
 * Ritz step (the batch queue of the QR iteration) gives up; the step then
 * ends and rigaqep_eigs returns RIGAQEP_ERR_TIMEOUT, leaving the CUDA
 * context usable.  Process-wide; 0 restores the default (2^22 polls, far
 * beyond any wait of a correct run).  Meant for failure-injection tests: a
 * limit of 1 makes the waits run out on any problem.  The waits of the TMA
 * copies are not affected (a copy must land before its CTA exits).
 * Defined by: no counterpart in the paper (failure reporting of the library). */
void rigaqep_set_wait_limit(uint32_t polls);

/* Thread-local message of the calling thread's last failed call ("" if none). */
const char* rigaqep_last_error(void);

/* Free the handle and every device buffer it owns (NULL is a no-op). */
void rigaqep_destroy(rigaqep_problem* prob);

#ifdef __cplusplus
}
#endif
#endif /* RIGAQEP_H */
