"""Python binding of the rigaqep C-ABI (argument marshalling only).

Every computation runs in ``_lib/librigaqep.so`` (CUDA, sm_103a); this module
only converts arguments, holds the handle and maps status codes to
exceptions.  PyTorch provides device buffers and the current stream.  There
is no fallback: if the library is missing or a call fails, an exception is
raised.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "librigaqep.so")

STATUS = {
    0: "OK", 1: "ERR_ARG", 2: "ERR_STATE", 3: "ERR_CUDA", 4: "ERR_OOM", 5: "ERR_PIVOT",
    6: "ERR_REFINEMENT", 7: "ERR_NO_CONVERGENCE", 8: "ERR_TIMEOUT", 9: "ERR_INTERNAL",
}

# every symbol declared in include/rigaqep.h
EXPORTS = [
    "rigaqep_assemble", "rigaqep_analyze", "rigaqep_factor", "rigaqep_solve", "rigaqep_eigs",
    "rigaqep_grad_damping", "rigaqep_grad_damping_noalloc", "rigaqep_export_csr", "rigaqep_export_symbolic", "rigaqep_get_info",
    "rigaqep_symbolic_create", "rigaqep_symbolic_sizes", "rigaqep_symbolic_export",
    "rigaqep_symbolic_counts",
    "rigaqep_symbolic_destroy", "rigaqep_last_error", "rigaqep_destroy", "rigaqep_batch_eigs",
    "rigaqep_front_gemm", "rigaqep_set_wait_limit", "rigaqep_inertia", "rigaqep_eigs_undamped",
    "rigaqep_factor_complex", "rigaqep_solve_complex",
]


FP64, TF32_IR, FP32_IR, BF16_IR = 0, 1, 2, 3   # rigaqep_precision


class RigaqepError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class MeshDesc(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in
                ("ne_x", "ne_y", "p", "block_x", "block_y", "n_quad", "leaf_min")]


class EigsOpts(ctypes.Structure):
    _fields_ = [("krylov_dim", ctypes.c_int32), ("max_restarts", ctypes.c_int32),
                ("tol", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("precision", ctypes.c_int32), ("shift_mode", ctypes.c_int32),
                ("shift", ctypes.c_double), ("ncand", ctypes.c_int32),
                ("scaling", ctypes.c_int32), ("shift_imag", ctypes.c_double)]


class BatchJob(ctypes.Structure):
    _fields_ = [("problem", ctypes.c_int32), ("neig", ctypes.c_int32), ("target", ctypes.c_double),
                ("opts", EigsOpts), ("lam", ctypes.c_void_p), ("X", ctypes.c_void_p),
                ("eta", ctypes.c_void_p), ("n_converged", ctypes.c_int32),
                ("status", ctypes.c_int32), ("certified", ctypes.c_int32),
                ("reused_candidates", ctypes.c_int32), ("eigs_ms", ctypes.c_double)]


class Info(ctypes.Structure):
    _fields_ = ([(n, ctypes.c_int64) for n in
                 ("n1", "N", "nnz", "nsuper", "nlevels", "nnz_L", "factor_flops", "max_front",
                  "n_apply", "n_restarts", "n_spmv", "n_vv", "n_qr_sweeps")]
                + [(n, ctypes.c_double) for n in
                   ("norm_K", "norm_M", "norm_C", "factor_ms", "eigs_ms", "fb_ms")]
                + [("certified", ctypes.c_int64), ("cert_margin", ctypes.c_double),
                   ("n_launches", ctypes.c_int64), ("ritz_ms", ctypes.c_double),
                   ("ritz_phase_cycles", ctypes.c_double * 6),
                   ("n_ir", ctypes.c_int64), ("ir_residual", ctypes.c_double),
                   ("reused_candidates", ctypes.c_int64), ("nnz_L_exact", ctypes.c_int64),
                   ("factor_flops_exact", ctypes.c_int64), ("scale_factor", ctypes.c_double),
                   ("tc_wide_levels", ctypes.c_int64)])

    def as_dict(self):
        d = {n: getattr(self, n) for n, _ in self._fields_}
        d["ritz_phase_cycles"] = list(self.ritz_phase_cycles)
        return d



_lib = None


def load():
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    P, I32, I64, D, V = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                         ctypes.c_void_p)
    sig = {
        "rigaqep_assemble": [ctypes.POINTER(MeshDesc), P, I32, V, ctypes.POINTER(P)],
        "rigaqep_analyze": [P],
        "rigaqep_factor": [P, D, I32],
        "rigaqep_solve": [P, P, P, I32, I32],
        "rigaqep_eigs": [P, I32, D, ctypes.POINTER(EigsOpts), P, P, P, P, ctypes.POINTER(I32)],
        "rigaqep_grad_damping": [P, I32, P, P, P],
        "rigaqep_grad_damping_noalloc": [P, I32, P, P, P],
        "rigaqep_export_csr": [P, P, P, P, P, P],
        "rigaqep_export_symbolic": [P, P, P, P, P, P, P],
        "rigaqep_get_info": [P, ctypes.POINTER(Info)],
        "rigaqep_symbolic_create": [ctypes.POINTER(MeshDesc), ctypes.POINTER(P)],
        "rigaqep_symbolic_sizes": [P, ctypes.POINTER(I64)],
        "rigaqep_symbolic_counts": [P, ctypes.POINTER(I64)],
        "rigaqep_symbolic_export": [P, P, P, P, P, P, P, P, P],
        "rigaqep_batch_eigs": [ctypes.POINTER(P), I32, ctypes.POINTER(BatchJob), I32, I32],
        "rigaqep_front_gemm": [I32, I32, I32, I32, P, P, P, V],
        "rigaqep_inertia": [P, D, ctypes.POINTER(I64)],
        "rigaqep_factor_complex": [P, D, D],
        "rigaqep_solve_complex": [P, P, P, I32],
        "rigaqep_eigs_undamped": [P, D, D, I32, ctypes.POINTER(EigsOpts), P, P, P, P,
                                  ctypes.POINTER(I32), ctypes.POINTER(I32), ctypes.POINTER(I32)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.rigaqep_symbolic_destroy.argtypes = [P]
    lib.rigaqep_symbolic_destroy.restype = None
    lib.rigaqep_destroy.argtypes = [P]
    lib.rigaqep_destroy.restype = None
    lib.rigaqep_set_wait_limit.argtypes = [ctypes.c_uint32]
    lib.rigaqep_set_wait_limit.restype = None
    lib.rigaqep_last_error.argtypes = []
    lib.rigaqep_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(code):
    if code != 0:
        raise RigaqepError(code, load().rigaqep_last_error().decode())


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(a.data_ptr())


def mesh_desc(ne, p, block, n_quad=0, leaf_min=0):
    return MeshDesc(ne, ne, p, block, block, n_quad, leaf_min)


def symbolic_host(ne, p, block, n_quad=0, leaf_min=0):
    """Pattern + symbolic phase on the host only (no CUDA call)."""
    lib = load()
    h = ctypes.c_void_p()
    md = mesh_desc(ne, p, block, n_quad, leaf_min)
    _check(lib.rigaqep_symbolic_create(ctypes.byref(md), ctypes.byref(h)))
    try:
        sz = (ctypes.c_int64 * 6)()
        _check(lib.rigaqep_symbolic_sizes(h, sz))
        N, nnz, ns, nu, nl, n1 = list(sz)
        out = dict(perm=np.empty(N, np.int32), sptr=np.empty(ns + 1, np.int32),
                   parent=np.empty(ns, np.int32), upd_ptr=np.empty(ns + 1, np.int32),
                   upd_idx=np.empty(nu, np.int32), level=np.empty(ns, np.int32),
                   rowptr=np.empty(N + 1, np.int32), col=np.empty(nnz, np.int32))
        _check(lib.rigaqep_symbolic_export(h, *[_ptr(out[k]) for k in
                                                ("perm", "sptr", "parent", "upd_ptr", "upd_idx",
                                                 "level", "rowptr", "col")]))
        out["nlevels"] = nl
        out["n1"] = n1
        cnt = (ctypes.c_int64 * 4)()
        _check(lib.rigaqep_symbolic_counts(h, cnt))
        out["nnz_L"], out["factor_flops"], out["nnz_L_exact"], out["factor_flops_exact"] = list(cnt)
        return out
    finally:
        lib.rigaqep_symbolic_destroy(h)


class Problem:
    """One rIGA QEP on the current CUDA device (owns its device memory)."""

    def __init__(self, ne, p, block, sigma_e, n_quad=0, leaf_min=0, stream=None):
        import torch
        self._torch = torch
        self.lib = load()
        self.ne, self.p, self.block = ne, p, block
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        if isinstance(sigma_e, np.ndarray):
            sig = np.ascontiguousarray(sigma_e, dtype=np.float64)
            on_dev = 0
        else:
            sig = sigma_e.contiguous().to(torch.float64)
            on_dev = 1 if sig.is_cuda else 0
        count = sig.size if isinstance(sig, np.ndarray) else sig.numel()
        if count != ne * ne:
            raise ValueError("sigma_e must have ne*ne entries")
        self._h = ctypes.c_void_p()
        md = mesh_desc(ne, p, block, n_quad, leaf_min)
        _check(self.lib.rigaqep_assemble(ctypes.byref(md), _ptr(sig), on_dev,
                                         ctypes.c_void_p(stream.cuda_stream), ctypes.byref(self._h)))
        inf = self.info()
        self.N, self.nnz, self.n1 = inf["N"], inf["nnz"], inf["n1"]

    # -- lifecycle
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self.lib.rigaqep_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- pipeline
    def analyze(self):
        _check(self.lib.rigaqep_analyze(self._h))
        return self

    def factor(self, sigma, precision=0):
        _check(self.lib.rigaqep_factor(self._h, float(sigma), precision))
        return self

    def solve(self, b, out=None, transpose=0):
        """x = Q(sigma)^{-1} b for a float64 CUDA tensor b of shape (N,) or (nrhs, N)."""
        torch = self._torch
        if b.dtype != torch.float64 or b.device.type != "cuda":
            raise ValueError("b must be a float64 CUDA tensor")
        if not ((b.dim() == 1 and b.shape[0] == self.N) or (b.dim() == 2 and b.shape[1] == self.N)):
            raise ValueError(f"b must have shape ({self.N},) or (nrhs, {self.N})")
        b = b.contiguous()
        nrhs = 1 if b.dim() == 1 else b.shape[0]
        if out is None:
            x = torch.empty_like(b)
        else:
            if (out.dtype != torch.float64 or out.device != b.device or not out.is_contiguous()
                    or tuple(out.shape) != tuple(b.shape)):
                raise ValueError("out must be a contiguous float64 tensor shaped and placed like b")
            x = out
        _check(self.lib.rigaqep_solve(self._h, _ptr(b), _ptr(x), nrhs, transpose))
        return x

    def eigs(self, neig, sigma, m=None, tol=1e-10, max_restarts=1000, seed=1, v1=None,
             raise_on_noconv=True, shift=None, ncand=None, precision=FP64, scaling=False):
        """Eigenpairs nearest the target sigma: (lambda (neig,) complex,
        X (neig, N) complex, eta (neig,), n_converged, status).

        shift=None places the spectral shift at sigma; a real shift selects
        the in-region mode (ncand pairs converged around the shift, the neig
        nearest sigma returned; see info()["certified"]).  precision=FP32_IR
        factorises in FP32 and refines every solve in FP64."""
        torch = self._torch
        dev = torch.device("cuda", torch.cuda.current_device())
        lam = torch.empty((neig, 2), dtype=torch.float64, device=dev)
        X = torch.empty((neig, self.N, 2), dtype=torch.float64, device=dev)
        eta = torch.empty(neig, dtype=torch.float64, device=dev)
        nconv = ctypes.c_int32(0)
        opts = eigs_opts(neig, m, tol, max_restarts, seed, shift, ncand, precision, scaling)
        if v1 is not None:
            v1 = v1.contiguous().to(device=dev, dtype=torch.float64)
            if v1.numel() != 2 * self.N:
                raise ValueError(f"v1 must have 2N = {2 * self.N} entries")
        st = self.lib.rigaqep_eigs(self._h, neig, float(sigma), ctypes.byref(opts), _ptr(v1),
                                   _ptr(lam), _ptr(X), _ptr(eta), ctypes.byref(nconv))
        if st != 0 and not (st == 7 and not raise_on_noconv):
            _check(st)
        return (torch.view_as_complex(lam), torch.view_as_complex(X), eta, nconv.value, st)

    def grad_damping(self, lam, X):
        """d lambda_k / d sigma_e, complex tensor of shape (neig, ne*ne)."""
        torch = self._torch
        if lam.dtype != torch.complex128 or X.dtype != torch.complex128:
            raise ValueError("lam and X must be complex128")
        if lam.dim() != 1 or X.dim() != 2 or X.shape[0] != lam.shape[0] or X.shape[1] != self.N:
            raise ValueError(f"need lam (neig,) and X (neig, {self.N})")
        if lam.device != X.device or lam.device.type != "cuda":
            raise ValueError("lam and X must be on one CUDA device")
        neig = lam.shape[0]
        lam_r = torch.view_as_real(lam.contiguous()).contiguous()
        X_r = torch.view_as_real(X.contiguous()).contiguous()
        G = torch.empty((neig, self.ne * self.ne, 2), dtype=torch.float64, device=lam.device)
        _check(self.lib.rigaqep_grad_damping(self._h, neig, _ptr(lam_r), _ptr(X_r), _ptr(G)))
        return torch.view_as_complex(G)

    def grad_damping_noalloc(self, lam, X, out=None):
        """Same as grad_damping, writing into the caller's buffer out (neig,
        ne*ne, 2 float64) with no device allocation inside the library call.
        lam (neig complex128) and X (neig x N complex128) must be on the
        device of out; every shape, dtype and device is checked here, since
        the library writes neig * ne^2 complex values through out."""
        torch = self._torch
        if lam.dtype != torch.complex128 or X.dtype != torch.complex128:
            raise ValueError("lam and X must be complex128")
        if lam.dim() != 1 or X.dim() != 2 or X.shape[0] != lam.shape[0] or X.shape[1] != self.N:
            raise ValueError(f"need lam (neig,) and X (neig, {self.N})")
        neig = lam.shape[0]
        lam_r = torch.view_as_real(lam.contiguous()).contiguous()
        X_r = torch.view_as_real(X.contiguous()).contiguous()
        if out is None:
            out = torch.empty((neig, self.ne * self.ne, 2), dtype=torch.float64, device=lam.device)
        if (out.dtype != torch.float64 or not out.is_contiguous()
                or tuple(out.shape) != (neig, self.ne * self.ne, 2)):
            raise ValueError(f"out must be a contiguous float64 tensor of shape "
                             f"({neig}, {self.ne * self.ne}, 2)")
        if not (out.device == lam.device == X.device) or out.device.type != "cuda":
            raise ValueError("lam, X and out must be on the same CUDA device")
        _check(self.lib.rigaqep_grad_damping_noalloc(self._h, neig, _ptr(lam_r), _ptr(X_r),
                                                     _ptr(out)))
        return torch.view_as_complex(out)

    # -- complex shift
    def factor_complex(self, s):
        """Complex symmetric LDL^T of Q(s) for a complex shift s."""
        _check(self.lib.rigaqep_factor_complex(self._h, float(s.real), float(s.imag)))
        return self

    def solve_complex(self, b):
        """x = Q(s)^{-1} b with the complex factor; b: complex128 CUDA tensor (N,)."""
        torch = self._torch
        if b.dim() != 1 or b.shape[0] != self.N or b.device.type != "cuda":
            raise ValueError(f"b must be a CUDA tensor of shape ({self.N},)")
        br = torch.view_as_real(b.contiguous().to(torch.complex128)).contiguous()
        x = torch.empty_like(br)
        _check(self.lib.rigaqep_solve_complex(self._h, _ptr(br), _ptr(x), 1))
        return torch.view_as_complex(x)

    # -- undamped pencil K x = mu M x
    def inertia(self, mu):
        """Number of eigenvalues of K x = mu' M x below mu (Sylvester)."""
        n = ctypes.c_int64(0)
        _check(self.lib.rigaqep_inertia(self._h, float(mu), ctypes.byref(n)))
        return n.value

    def eigs_undamped(self, mu_lo, mu_hi, nmax=90, m=None, tol=1e-10, max_restarts=1000, seed=1,
                      v1=None):
        """Eigenpairs of K x = mu M x with mu in [mu_lo, mu_hi):
        (mu (n,), X (n, N) real, resid (n,), count, certified)."""
        torch = self._torch
        dev = torch.device("cuda", torch.cuda.current_device())
        mu = torch.empty(max(nmax, 1), dtype=torch.float64, device=dev)
        X = torch.empty((max(nmax, 1), self.N), dtype=torch.float64, device=dev)
        res = torch.empty(max(nmax, 1), dtype=torch.float64, device=dev)
        opts = eigs_opts(1, m or 0, tol, max_restarts, seed)
        opts.krylov_dim = m or 0
        if v1 is not None:
            v1 = v1.contiguous().to(device=dev, dtype=torch.float64)
            if v1.numel() != self.N:
                raise ValueError(f"v1 must have N = {self.N} entries")
        nf, cnt, cert = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
        _check(self.lib.rigaqep_eigs_undamped(self._h, float(mu_lo), float(mu_hi), int(nmax),
                                              ctypes.byref(opts), _ptr(v1), _ptr(mu), _ptr(X),
                                              _ptr(res), ctypes.byref(nf), ctypes.byref(cnt),
                                              ctypes.byref(cert)))
        n = nf.value
        return mu[:n], X[:n], res[:n], cnt.value, cert.value

    # -- introspection
    def info(self):
        inf = Info()
        _check(self.lib.rigaqep_get_info(self._h, ctypes.byref(inf)))
        return inf.as_dict()

    def export_csr(self):
        N, nnz = self.N, self.nnz
        out = dict(rowptr=np.empty(N + 1, np.int32), col=np.empty(nnz, np.int32),
                   K=np.empty(nnz), M=np.empty(nnz), C=np.empty(nnz))
        _check(self.lib.rigaqep_export_csr(self._h, *[_ptr(out[k]) for k in
                                                      ("rowptr", "col", "K", "M", "C")]))
        return out

    def export_symbolic(self):
        inf = self.info()
        ns = inf["nsuper"]
        out = dict(perm=np.empty(self.N, np.int32), sptr=np.empty(ns + 1, np.int32),
                   parent=np.empty(ns, np.int32), upd_ptr=np.empty(ns + 1, np.int32),
                   level=np.empty(ns, np.int32))
        _check(self.lib.rigaqep_export_symbolic(self._h, _ptr(out["perm"]), _ptr(out["sptr"]),
                                                _ptr(out["parent"]), _ptr(out["upd_ptr"]), None,
                                                _ptr(out["level"])))
        out["upd_idx"] = np.empty(int(out["upd_ptr"][-1]), np.int32)
        _check(self.lib.rigaqep_export_symbolic(self._h, None, None, None, None,
                                                _ptr(out["upd_idx"]), None))
        return out


def eigs_opts(neig, m=None, tol=1e-10, max_restarts=1000, seed=1, shift=None, ncand=None,
              precision=FP64, scaling=False):
    """rigaqep_eigs_opts with the defaults of Problem.eigs."""
    if isinstance(shift, complex):   # complex shift: the neig eigenvalues nearest it
        nc = 2 * neig + 4 if ncand is None else ncand
        m = m or min(96, 2 * nc + 20)
        return EigsOpts(m, max_restarts, tol, seed, precision, 2, shift.real, nc,
                        1 if scaling else 0, shift.imag)
    nc = neig if ncand is None else ncand
    m = m or min(96, 2 * nc + 20)
    return EigsOpts(m, max_restarts, tol, seed, precision, 0 if shift is None else 1,
                    0.0 if shift is None else float(shift), nc, 1 if scaling else 0, 0.0)


def batch_eigs(problems, jobs, nthreads=0, raise_on_error=True):
    """Run many eigensolves over many Problems in one rigaqep_batch_eigs call.

    jobs: list of dicts with keys problem (index into problems), neig, target
    and optionally m, tol, max_restarts, seed, shift, ncand (as Problem.eigs;
    the start vector is the seeded one).  Returns one dict per job: lam
    (neig,) complex, X (neig, N) complex, eta (neig,), n_converged, status,
    certified, reused_candidates, eigs_ms.  Problems on distinct streams run
    concurrently."""
    import torch
    lib = load()
    dev = torch.device("cuda", torch.cuda.current_device())
    handles = (ctypes.c_void_p * len(problems))(*[pr._h.value for pr in problems])
    arr = (BatchJob * len(jobs))()
    outs = []
    for j, d in enumerate(jobs):
        pr = problems[d["problem"]]
        neig = d["neig"]
        lam = torch.empty((neig, 2), dtype=torch.float64, device=dev)
        X = torch.empty((neig, pr.N, 2), dtype=torch.float64, device=dev)
        eta = torch.empty(neig, dtype=torch.float64, device=dev)
        opts = eigs_opts(neig, **{k: d[k] for k in ("m", "tol", "max_restarts", "seed", "shift",
                                                   "ncand", "precision", "scaling") if k in d})
        arr[j] = BatchJob(d["problem"], neig, float(d["target"]), opts, lam.data_ptr(),
                          X.data_ptr(), eta.data_ptr(), 0, 0, 0, 0, 0.0)
        outs.append((lam, X, eta))
    # the handles' streams must see the caller's pending work (e.g. output allocation)
    torch.cuda.current_stream().synchronize()
    code = lib.rigaqep_batch_eigs(handles, len(problems), arr, len(jobs), int(nthreads))
    if code != 0 and raise_on_error:
        _check(code)
    res = []
    for j, (lam, X, eta) in enumerate(outs):
        J = arr[j]
        res.append(dict(lam=torch.view_as_complex(lam), X=torch.view_as_complex(X), eta=eta,
                        n_converged=J.n_converged, status=J.status, certified=J.certified,
                        reused_candidates=J.reused_candidates, eigs_ms=J.eigs_ms))
    return res


def front_gemm(A, B, precision=TF32_IR, stream=None):
    """C = A B^T on the tensor cores through the front factorisation's
    staging and tcgen05 kernels (rigaqep_front_gemm); A (m x k), B (n x k):
    contiguous float32 CUDA tensors.  Returns C (m x n float32)."""
    import torch
    if A.dtype != torch.float32 or B.dtype != torch.float32:
        raise ValueError("A and B must be float32")
    if A.dim() != 2 or B.dim() != 2 or A.shape[1] != B.shape[1]:
        raise ValueError("need A (m x k) and B (n x k)")
    if A.device.type != "cuda" or B.device != A.device:
        raise ValueError("A and B must be on one CUDA device")
    A, B = A.contiguous(), B.contiguous()
    m, k = A.shape
    n = B.shape[0]
    C = torch.empty((m, n), dtype=torch.float32, device=A.device)
    st = stream if stream is not None else torch.cuda.current_stream(A.device)
    _check(load().rigaqep_front_gemm(precision, m, n, k, _ptr(A), _ptr(B), _ptr(C),
                                     ctypes.c_void_p(st.cuda_stream)))
    return C
