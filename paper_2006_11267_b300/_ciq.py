"""ctypes binding of libciq (include/ciq.h): argument marshalling only.

Every function here has the name of the C entry point it calls.  Arrays may be
CUDA torch tensors (device pointers, launched on the current torch stream),
CPU torch tensors or NumPy arrays (host pointers: the library copies them to
and from the device inside the call).  Nothing is computed here.

Layouts (see include/ciq.h): X is (N, d) row-major; right-hand sides are
passed as a (T, N) array whose row c is right-hand side c (the C layout
"T columns of N entries").
"""
from __future__ import annotations

import ctypes
import dataclasses
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libciq.so")

CIQ_MAX_DIM = 16
CIQ_MAX_Q = 32

STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "out of device memory",
          4: "not converged within max_iter", 5: "non-finite Lanczos coefficient",
          6: "unsupported option", 7: "problem exceeds the static scratch of the allocation-free entry point",
          8: "a bounded wait of the tensor-core MVM gave up"}
(CIQ_OK, CIQ_ERR_ARG, CIQ_ERR_CUDA, CIQ_ERR_NOMEM, CIQ_NOT_CONVERGED, CIQ_ERR_NAN, CIQ_ERR_UNSUPPORTED,
 CIQ_ERR_SCRATCH_TOO_SMALL, CIQ_ERR_TIMEOUT) = range(9)

KERNELS = {"rbf": 0, "matern52": 1}
PRECISIONS = {"fp32": 0, "tf32": 1, "bf16": 2, "fp16": 3}
MVM_MODES = {"auto": 0, "onthefly": 1, "stored": 2}
STOP_RULES = {"residual": 0, "errbound": 1}
SQRT_FORMS = {"identity": 0, "mvm": 1}
KRYLOV_FORMS = {"auto": 0, "recurrence": 1, "basis": 2}


class CiqError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {STATUS.get(status, status)} (status {status})")
        self.status = status


class _Kernel(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("lengthscale", ctypes.c_double),
                ("outputscale", ctypes.c_double), ("noise", ctypes.c_double)]


class _Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("mvm", ctypes.c_int), ("stop_rule", ctypes.c_int),
                ("sqrt_form", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("lanczos_iters", ctypes.c_int), ("check_every", ctypes.c_int),
                ("profile", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("lanczos_start", ctypes.c_void_p), ("lmax_margin", ctypes.c_double),
                ("lmin_div", ctypes.c_double), ("lmin", ctypes.c_double), ("lmax", ctypes.c_double),
                ("quad_w", ctypes.c_void_p), ("quad_t", ctypes.c_void_p),
                ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t), ("graph", ctypes.c_int),
                ("tc_split", ctypes.c_int), ("fault_inject", ctypes.c_int), ("krylov", ctypes.c_int),
                ("batch_split_rows", ctypes.c_int), ("batch_split", ctypes.c_int), ("precond_rank", ctypes.c_int)]


class _Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("iters_min", ctypes.c_int), ("converged", ctypes.c_int),
                ("lanczos_iters", ctypes.c_int), ("resid_max", ctypes.c_double),
                ("errbound_max", ctypes.c_double), ("ritz_min", ctypes.c_double),
                ("ritz_max", ctypes.c_double), ("lmin_used", ctypes.c_double),
                ("lmax_used", ctypes.c_double), ("w", ctypes.c_double * CIQ_MAX_Q),
                ("t", ctypes.c_double * CIQ_MAX_Q), ("q", ctypes.c_int), ("launches", ctypes.c_int),
                ("t_total_ms", ctypes.c_double), ("t_prepass_ms", ctypes.c_double),
                ("t_mvm_ms", ctypes.c_double), ("t_step_ms", ctypes.c_double),
                ("mvm_launches", ctypes.c_int), ("step_launches", ctypes.c_int),
                ("ritz_max_solve", ctypes.c_double), ("krylov", ctypes.c_int), ("precond_rank", ctypes.c_int)]


class _Problem(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("N", ctypes.c_int64), ("d", ctypes.c_int), ("kern", _Kernel),
                ("B", ctypes.c_void_p), ("T", ctypes.c_int), ("out", ctypes.c_void_p),
                ("lmin", ctypes.c_double), ("lmax", ctypes.c_double)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libciq.so (built in-tree).  Raises if it is missing: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing; build it with `python -m paper_2006_11267_b300.build`")
    L = ctypes.CDLL(LIB_PATH)
    P, I, I64, D, U64, S = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double,
                            ctypes.c_uint64, ctypes.c_size_t)
    KP, OP, IP = ctypes.POINTER(_Kernel), ctypes.POINTER(_Options), ctypes.POINTER(_Info)
    DP = ctypes.POINTER(ctypes.c_double)
    sig = {
        "ciq_status_string": (ctypes.c_char_p, [I]),
        "ciq_default_options": (None, [OP]),
        "ciq_quad_nodes": (I, [D, D, I, DP, DP]),
        "ciq_lanczos_bounds": (I, [P, I64, I, KP, I, U64, P, DP, DP, DP, DP, P]),
        "ciq_sqrt": (I, [P, I64, I, KP, P, I, I, D, OP, P, IP, P]),
        "ciq_invsqrt": (I, [P, I64, I, KP, P, I, I, D, OP, P, IP, P]),
        "ciq_sqrt_f64": (I, [P, I64, I, KP, P, I, I, D, OP, P, IP, P]),
        "ciq_invsqrt_f64": (I, [P, I64, I, KP, P, I, I, D, OP, P, IP, P]),
        "ciq_kernel_mvm": (I, [P, I64, I, KP, P, I, P, I, P]),
        "ciq_kernel_mvm_f64": (I, [P, I64, I, KP, P, I, P, P]),
        "ciq_kernel_matrix": (I, [P, I64, I, KP, P, I64, P]),
        "ciq_stored_mvm": (I, [P, I64, I64, P, I, P, I, P]),
        "ciq_sqrt_dense": (I, [P, I64, I64, P, I, I, D, OP, P, IP, P]),
        "ciq_invsqrt_vjp": (I, [P, I64, I, KP, P, P, I, I, D, OP, P, P, DP, IP, P]),
        "ciq_sqrt_vjp": (I, [P, I64, I, KP, P, P, I, I, D, OP, P, P, DP, IP, P]),
        "ciq_invsqrt_dense": (I, [P, I64, I64, P, I, I, D, OP, P, IP, P]),
        "ciq_workspace_bytes": (S, [I64, I, I, I, OP]),
        "ciq_kernel_mvm_noalloc": (I, [P, I64, I, KP, P, I, P, P]),
        "ciq_noalloc_scratch_floats": (S, []),
        "ciq_sqrt_batched": (I, [ctypes.POINTER(_Problem), I, I, D, OP, IP, P]),
        "ciq_invsqrt_batched": (I, [ctypes.POINTER(_Problem), I, I, D, OP, IP, P]),
        "ciq_sqrt_batched_learned": (I, [ctypes.POINTER(_Problem), I, I, D, OP, P, D, IP, P, P]),
        "ciq_invsqrt_batched_learned": (I, [ctypes.POINTER(_Problem), I, I, D, OP, P, D, IP, P, P]),
        "ciq_mlp_features": (I, [ctypes.POINTER(_Problem), I, P, P]),
        "ciq_mlp_normaliser": (I, [P, P, I, P, P]),
        "ciq_mlp_init": (I, [P, U64, P]),
        "ciq_mlp_loss_grad": (I, [P, P, P, I, DP, P, P]),
        "ciq_mlp_train": (I, [P, P, P, P, I, I, I, ctypes.c_float, U64, I, P, P]),
        "ciq_mlp_predict": (I, [P, P, I, P, I, P]),
        "ciq_sqrt_precond": (I, [P, I64, I, KP, I, P, I64, P, I, I, D, OP, P, IP, P]),
        "ciq_invsqrt_precond": (I, [P, I64, I, KP, I, P, I64, P, I, I, D, OP, P, IP, P]),
        "ciq_pivoted_cholesky": (I, [P, I64, I, KP, I, P, I64, P, ctypes.POINTER(I), P]),
        "ciq_precond_workspace_bytes": (S, [I64, I, I, I, I, OP]),
        "ciq_posterior_sample": (I, [P, I64, P, P, I64, I, I, DP, D, D, D, D, P, I, I, D, OP, P, IP, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


@dataclasses.dataclass
class Kernel:
    """Kernel type and hyperparameters; ``noise`` is sigma^2 on the diagonal."""
    type: str = "rbf"
    lengthscale: float = 1.0
    outputscale: float = 1.0
    noise: float = 0.0

    def c(self) -> _Kernel:
        return _Kernel(KERNELS[self.type], float(self.lengthscale), float(self.outputscale),
                       float(self.noise))


# ------------------------------------------------------------ marshalling ---
def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """Pointer of a contiguous torch tensor or NumPy array (None -> NULL)."""
    if x is None:
        return None
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr())
    if not x.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return ctypes.c_void_p(x.ctypes.data)


def _stream(*arrays):
    for a in arrays:
        if a is not None and _is_torch(a) and a.is_cuda:
            import torch
            return ctypes.c_void_p(torch.cuda.current_stream(a.device).cuda_stream)
    return None


def _empty_like_rhs(B, dtype):
    if _is_torch(B):
        return B.new_empty(B.shape)
    return np.empty(B.shape, dtype=dtype)


def make_options(**kw) -> _Options:
    o = _Options()
    lib().ciq_default_options(ctypes.byref(o))
    keep = []
    for k, v in kw.items():
        if v is None:
            continue
        if k == "precision":
            o.precision = PRECISIONS[v] if isinstance(v, str) else int(v)
        elif k == "mvm":
            o.mvm = MVM_MODES[v] if isinstance(v, str) else int(v)
        elif k == "stop_rule":
            o.stop_rule = STOP_RULES[v] if isinstance(v, str) else int(v)
        elif k == "sqrt_form":
            o.sqrt_form = SQRT_FORMS[v] if isinstance(v, str) else int(v)
        elif k == "krylov":
            o.krylov = KRYLOV_FORMS[v] if isinstance(v, str) else int(v)
        elif k in ("lanczos_start", "workspace"):
            setattr(o, k, _ptr(v))
            keep.append(v)
        elif k == "nodes":
            w = np.ascontiguousarray(v[0], dtype=np.float64)
            t = np.ascontiguousarray(v[1], dtype=np.float64)
            o.quad_w, o.quad_t = w.ctypes.data, t.ctypes.data
            keep += [w, t]
        else:
            setattr(o, k, v)
    o._keep = keep
    return o


def _info_dict(info: _Info, status: int) -> dict:
    q = info.q
    return dict(status=status, status_name=STATUS.get(status), iters=info.iters,
                iters_min=info.iters_min, converged=info.converged,
                lanczos_iters=info.lanczos_iters, resid_max=info.resid_max,
                errbound_max=info.errbound_max, ritz_min=info.ritz_min, ritz_max=info.ritz_max,
                lmin_used=info.lmin_used, lmax_used=info.lmax_used,
                w=np.array(info.w[:q]), t=np.array(info.t[:q]), launches=info.launches,
                t_total_ms=info.t_total_ms, t_prepass_ms=info.t_prepass_ms, t_mvm_ms=info.t_mvm_ms,
                t_step_ms=info.t_step_ms, mvm_launches=info.mvm_launches,
                step_launches=info.step_launches, ritz_max_solve=info.ritz_max_solve,
                krylov={v: k for k, v in KRYLOV_FORMS.items()}.get(info.krylov),
                precond_rank=info.precond_rank)


def _check(status: int, where: str, allow=(CIQ_OK, CIQ_NOT_CONVERGED)):
    if status not in allow:
        raise CiqError(status, where)


def _solve(name, X, kernel: Kernel, B, Q, tol, out=None, **opts):
    N, d = X.shape
    T = B.shape[0]
    if B.shape[1] != N:
        raise ValueError("B must have shape (T, N)")
    fp64 = name.endswith("_f64")
    if out is None:
        out = _empty_like_rhs(B, np.float64 if fp64 else np.float32)
    o = make_options(**opts)
    info = _Info()
    k = kernel.c()
    st = getattr(lib(), name)(_ptr(X), N, d, ctypes.byref(k), _ptr(B), T, int(Q), float(tol),
                              ctypes.byref(o), _ptr(out), ctypes.byref(info), _stream(X, B, out))
    _check(st, name)
    return out, _info_dict(info, st)


def ciq_sqrt(X, kernel, B, Q, tol=0.0, out=None, **opts):
    """K^{1/2} B (FP32 vectors, FP64 scalars). Returns (out, info)."""
    return _solve("ciq_sqrt", X, kernel, B, Q, tol, out, **opts)


def ciq_invsqrt(X, kernel, B, Q, tol=0.0, out=None, **opts):
    """K^{-1/2} B (FP32 vectors, FP64 scalars). Returns (out, info)."""
    return _solve("ciq_invsqrt", X, kernel, B, Q, tol, out, **opts)


def ciq_sqrt_f64(X, kernel, B, Q, tol=0.0, out=None, **opts):
    """K^{1/2} B in FP64 end to end. Returns (out, info)."""
    return _solve("ciq_sqrt_f64", X, kernel, B, Q, tol, out, **opts)


def ciq_invsqrt_f64(X, kernel, B, Q, tol=0.0, out=None, **opts):
    """K^{-1/2} B in FP64 end to end. Returns (out, info)."""
    return _solve("ciq_invsqrt_f64", X, kernel, B, Q, tol, out, **opts)


def ciq_quad_nodes(lmin, lmax, Q):
    """(w, t) float64 arrays of length Q from the library's host routine."""
    w = np.zeros(Q)
    t = np.zeros(Q)
    DP = ctypes.POINTER(ctypes.c_double)
    st = lib().ciq_quad_nodes(float(lmin), float(lmax), int(Q), w.ctypes.data_as(DP), t.ctypes.data_as(DP))
    _check(st, "ciq_quad_nodes", allow=(CIQ_OK,))
    return w, t


def ciq_lanczos_bounds(X, kernel, iters=10, seed=0x5eed, start=None):
    """dict(ritz_min, ritz_max, lmin_used, lmax_used) from the device pre-pass."""
    N, d = X.shape
    vals = [ctypes.c_double() for _ in range(4)]
    k = kernel.c()
    st = lib().ciq_lanczos_bounds(_ptr(X), N, d, ctypes.byref(k), int(iters), int(seed), _ptr(start),
                                  *[ctypes.byref(v) for v in vals], _stream(X, start))
    _check(st, "ciq_lanczos_bounds", allow=(CIQ_OK,))
    return dict(zip(["ritz_min", "ritz_max", "lmin_used", "lmax_used"], [v.value for v in vals]))


def ciq_kernel_mvm(X, kernel, V, out=None, precision="fp32"):
    """(K_XX + sigma^2 I) V for device tensors; V and out are (T, N)."""
    N, d = X.shape
    T = V.shape[0]
    if out is None:
        out = V.new_empty(V.shape)
    k = kernel.c()
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    st = lib().ciq_kernel_mvm(_ptr(X), N, d, ctypes.byref(k), _ptr(V), T, _ptr(out), prec, _stream(X, V, out))
    _check(st, "ciq_kernel_mvm", allow=(CIQ_OK,))
    return out


def ciq_kernel_mvm_f64(X, kernel, V, out=None):
    N, d = X.shape
    T = V.shape[0]
    if out is None:
        out = V.new_empty(V.shape)
    k = kernel.c()
    st = lib().ciq_kernel_mvm_f64(_ptr(X), N, d, ctypes.byref(k), _ptr(V), T, _ptr(out), _stream(X, V, out))
    _check(st, "ciq_kernel_mvm_f64", allow=(CIQ_OK,))
    return out


def ciq_kernel_matrix(X, kernel, Kmat):
    N, d = X.shape
    k = kernel.c()
    st = lib().ciq_kernel_matrix(_ptr(X), N, d, ctypes.byref(k), _ptr(Kmat), Kmat.shape[1], _stream(X, Kmat))
    _check(st, "ciq_kernel_matrix", allow=(CIQ_OK,))
    return Kmat


def ciq_stored_mvm(Kmat, V, out=None, n=None, precision="fp32"):
    """Kmat V for a matrix in the layout ciq_kernel_matrix writes
    (round_up(N,128) rows of ldk floats); V and out are (T, N).  precision
    "fp16"/"bf16": tensor cores (split operands)."""
    N = V.shape[1] if n is None else n
    T = V.shape[0]
    if out is None:
        out = V.new_empty(V.shape)
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    st = lib().ciq_stored_mvm(_ptr(Kmat), N, Kmat.shape[1], _ptr(V), T, _ptr(out), prec, _stream(Kmat, V, out))
    _check(st, "ciq_stored_mvm", allow=(CIQ_OK,))
    return out


def _solve_precond(name, X, kernel, B, Q, tol, rank, L, out, **opts):
    N, d = X.shape
    T = B.shape[0]
    if B.shape[1] != N:
        raise ValueError("B must have shape (T, N)")
    ldl = N
    if L is not None:
        if L.ndim != 2 or L.shape[1] < N:
            raise ValueError("L must have shape (rank, ldl) with ldl >= N (row m is column m of the factor)")
        rank, ldl = L.shape
    if out is None:
        out = _empty_like_rhs(B, np.float32)
    o = make_options(**opts)
    info = _Info()
    k = kernel.c()
    st = getattr(lib(), name)(_ptr(X), N, d, ctypes.byref(k), int(rank), _ptr(L), int(ldl), _ptr(B), T, int(Q),
                              float(tol), ctypes.byref(o), _ptr(out), ctypes.byref(info), _stream(X, B, out, L))
    _check(st, name)
    return out, _info_dict(info, st)


def ciq_sqrt_precond(X, kernel, B, Q, tol=0.0, rank=100, L=None, out=None, **opts):
    """R B with R R^T = K (pivoted-Cholesky preconditioner of the given rank,
    or the caller's factor L of shape (rank, N)). Returns (out, info)."""
    return _solve_precond("ciq_sqrt_precond", X, kernel, B, Q, tol, rank, L, out, **opts)


def ciq_invsqrt_precond(X, kernel, B, Q, tol=0.0, rank=100, L=None, out=None, **opts):
    """R' B with R' R'^T = K^{-1} (see ciq_sqrt_precond). Returns (out, info)."""
    return _solve_precond("ciq_invsqrt_precond", X, kernel, B, Q, tol, rank, L, out, **opts)


def ciq_pivoted_cholesky(X, kernel, rank):
    """Partial pivoted Cholesky factor of K_XX: (L of shape (rank, N), pivots
    (int64, rank), columns formed).  Host arrays are returned for host X,
    device tensors for a device X."""
    N, d = X.shape
    if _is_torch(X):
        import torch
        L = torch.empty((rank, N), dtype=torch.float32, device=X.device)
        piv = torch.empty(rank, dtype=torch.int64, device=X.device)
    else:
        L = np.empty((rank, N), np.float32)
        piv = np.empty(rank, np.int64)
    got = ctypes.c_int()
    k = kernel.c()
    st = lib().ciq_pivoted_cholesky(_ptr(X), N, d, ctypes.byref(k), int(rank), _ptr(L), N, _ptr(piv),
                                    ctypes.byref(got), _stream(X, L, piv))
    _check(st, "ciq_pivoted_cholesky", allow=(CIQ_OK,))
    return L, piv, got.value


def ciq_posterior_sample(Xtr, y, Xc, kind, lengthscales, outputscale, noise, jitter, mean, eps, Q, tol=0.0,
                         out=None, **opts):
    """Posterior draws mu* + COV*^{1/2} eps at the candidates Xc (Nc, d) given
    training data Xtr (n, d), y (n,); eps and out are (T, Nc).  ARD
    lengthscales (d values). Returns (out, info)."""
    Nc, d = Xc.shape
    n = 0 if Xtr is None else Xtr.shape[0]
    T = eps.shape[0]
    if eps.shape[1] != Nc:
        raise ValueError("eps must have shape (T, Nc)")
    ls = np.ascontiguousarray(np.broadcast_to(np.asarray(lengthscales, dtype=np.float64), (d,)))
    if out is None:
        out = _empty_like_rhs(eps, np.float32)
    o = make_options(**opts)
    info = _Info()
    st = lib().ciq_posterior_sample(_ptr(Xtr), int(n), _ptr(y), _ptr(Xc), int(Nc), int(d), KERNELS[kind],
                                    ls.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(outputscale),
                                    float(noise), float(jitter), float(mean), _ptr(eps), int(T), int(Q), float(tol),
                                    ctypes.byref(o), _ptr(out), ctypes.byref(info), _stream(Xtr, Xc, eps, out))
    _check(st, "ciq_posterior_sample")
    return out, _info_dict(info, st)


def ciq_precond_workspace_bytes(N, d, T, Q, rank, **opts):
    o = make_options(**opts)
    return int(lib().ciq_precond_workspace_bytes(int(N), int(d), int(T), int(Q), int(rank), ctypes.byref(o)))


def _solve_dense(name, K, B, Q, tol, out=None, **opts):
    N = K.shape[0]
    if K.ndim != 2 or K.shape[1] < N:
        raise ValueError("K must have shape (N, ldk) with ldk >= N")
    T = B.shape[0]
    if B.shape[1] != N:
        raise ValueError("B must have shape (T, N)")
    if out is None:
        out = _empty_like_rhs(B, np.float32)
    o = make_options(**opts)
    info = _Info()
    st = getattr(lib(), name)(_ptr(K), N, K.shape[1], _ptr(B), T, int(Q), float(tol), ctypes.byref(o), _ptr(out),
                              ctypes.byref(info), _stream(K, B, out))
    _check(st, name)
    return out, _info_dict(info, st)


def ciq_sqrt_dense(K, B, Q, tol=0.0, out=None, **opts):
    """K^{1/2} B for an explicit SPD matrix K (N x N, FP32, row-major). Returns (out, info)."""
    return _solve_dense("ciq_sqrt_dense", K, B, Q, tol, out, **opts)


def ciq_invsqrt_dense(K, B, Q, tol=0.0, out=None, **opts):
    """K^{-1/2} B for an explicit SPD matrix K (N x N, FP32, row-major). Returns (out, info)."""
    return _solve_dense("ciq_invsqrt_dense", K, B, Q, tol, out, **opts)


def _vjp(name, X, kernel, B, G, Q, tol, **opts):
    N, d = X.shape
    T = B.shape[0]
    if B.shape != (T, N) or G.shape != (T, N):
        raise ValueError("B and G must have shape (T, N)")
    out = _empty_like_rhs(B, np.float32)
    grad_B = _empty_like_rhs(B, np.float32)
    grad = (ctypes.c_double * 3)()
    o = make_options(**opts)
    info = _Info()
    k = kernel.c()
    st = getattr(lib(), name)(_ptr(X), N, d, ctypes.byref(k), _ptr(B), _ptr(G), T, int(Q), float(tol),
                              ctypes.byref(o), _ptr(out), _ptr(grad_B), grad, ctypes.byref(info),
                              _stream(X, B, G))
    _check(st, name)
    return out, grad_B, np.array(grad[:]), _info_dict(info, st)


def ciq_invsqrt_vjp(X, kernel, B, G, Q, tol=0.0, **opts):
    """K^{-1/2} B and the gradients of sum(G * K^{-1/2} B) w.r.t. B and
    (lengthscale, outputscale, noise).  Returns (out, grad_B, grad_theta, info)."""
    return _vjp("ciq_invsqrt_vjp", X, kernel, B, G, Q, tol, **opts)


def ciq_sqrt_vjp(X, kernel, B, G, Q, tol=0.0, **opts):
    """K^{1/2} B and the gradients of sum(G * K^{1/2} B) w.r.t. B and
    (lengthscale, outputscale, noise).  Returns (out, grad_B, grad_theta, info)."""
    return _vjp("ciq_sqrt_vjp", X, kernel, B, G, Q, tol, **opts)


def ciq_workspace_bytes(N, d, T, Q, **opts):
    o = make_options(**opts)
    return int(lib().ciq_workspace_bytes(int(N), int(d), int(T), int(Q), ctypes.byref(o)))


def ciq_kernel_mvm_noalloc(X, kernel, V, out=None):
    """(K_XX + sigma^2 I) V through the allocation-free entry point.

    For callers that cannot allocate device memory: the library's scratch is
    a static device array (see include/ciq.h); ``out`` must be preallocated
    by such a caller.  V and out are (T, N) device tensors.
    """
    N, d = X.shape
    T = V.shape[0]
    if out is None:
        out = V.new_empty(V.shape)
    k = kernel.c()
    st = lib().ciq_kernel_mvm_noalloc(_ptr(X), N, d, ctypes.byref(k), _ptr(V), T, _ptr(out), _stream(X, V, out))
    _check(st, "ciq_kernel_mvm_noalloc", allow=(CIQ_OK,))
    return out


CIQ_MLP_INPUTS = 38
CIQ_MLP_OUTPUTS = 3
CIQ_MLP_PARAMS = 6933


def _problem_array(problems, need_b=True):
    P = len(problems)
    arr = (_Problem * P)()
    outs = []
    for i, pr in enumerate(problems):
        X = pr["X"]
        N, d = X.shape
        arr[i].X = _ptr(X).value
        arr[i].N = N
        arr[i].d = d
        arr[i].kern = pr["kernel"].c()
        arr[i].lmin = float(pr.get("lmin") or 0.0)
        arr[i].lmax = float(pr.get("lmax") or 0.0)
        if not need_b:
            continue
        B = pr["B"]
        if B.shape[1] != N:
            raise ValueError("B must have shape (T, N)")
        out = pr.get("out")
        if out is None:
            out = _empty_like_rhs(B, np.float32)
        outs.append(out)
        arr[i].B = _ptr(B).value
        arr[i].T = B.shape[0]
        arr[i].out = _ptr(out).value
    return arr, outs


def _solve_batched(name, problems, Q, tol, **opts):
    """problems: sequence of dicts with X (N, d), kernel (Kernel), B (T, N)
    device tensors, optional out (T, N) and optional lmin, lmax."""
    P = len(problems)
    arr, outs = _problem_array(problems)
    o = make_options(**opts)
    infos = (_Info * P)()
    first = problems[0]
    st = getattr(lib(), name)(arr, P, int(Q), float(tol), ctypes.byref(o), infos,
                              _stream(first["X"], first["B"]))
    _check(st, name)
    return outs, [_info_dict(infos[i], st) for i in range(P)]


def ciq_sqrt_batched(problems, Q, tol=0.0, **opts):
    """K_p^{1/2} B_p for every problem of the batch. Returns (outs, infos)."""
    return _solve_batched("ciq_sqrt_batched", problems, Q, tol, **opts)


def ciq_invsqrt_batched(problems, Q, tol=0.0, **opts):
    """K_p^{-1/2} B_p for every problem of the batch. Returns (outs, infos)."""
    return _solve_batched("ciq_invsqrt_batched", problems, Q, tol, **opts)


def _solve_batched_learned(name, problems, Q, tol, theta, margin=0.0, **opts):
    P = len(problems)
    arr, outs = _problem_array(problems)
    o = make_options(**opts)
    infos = (_Info * P)()
    fb = (ctypes.c_int * P)()
    first = problems[0]
    st = getattr(lib(), name)(arr, P, int(Q), float(tol), ctypes.byref(o), _ptr(theta), float(margin), infos, fb,
                              _stream(first["X"], first["B"], theta))
    _check(st, name)
    res = [_info_dict(infos[i], st) for i in range(P)]
    for i in range(P):
        res[i]["fallback"] = int(fb[i])
    return outs, res


def ciq_sqrt_batched_learned(problems, Q, tol, theta, margin=0.0, **opts):
    """K_p^{1/2} B_p with bounds from the trained network ``theta`` (device,
    CIQ_MLP_PARAMS floats); infos carry ``fallback`` per problem."""
    return _solve_batched_learned("ciq_sqrt_batched_learned", problems, Q, tol, theta, margin, **opts)


def ciq_invsqrt_batched_learned(problems, Q, tol, theta, margin=0.0, **opts):
    """K_p^{-1/2} B_p with bounds from the trained network (see ciq_sqrt_batched_learned)."""
    return _solve_batched_learned("ciq_invsqrt_batched_learned", problems, Q, tol, theta, margin, **opts)


def ciq_mlp_features(problems, out=None):
    """(P, 38) device tensor of network inputs; problems need X and kernel."""
    import torch
    arr, _ = _problem_array(problems, need_b=False)
    X0 = problems[0]["X"]
    if out is None:
        out = torch.empty((len(problems), CIQ_MLP_INPUTS), dtype=torch.float32, device=X0.device)
    st = lib().ciq_mlp_features(arr, len(problems), _ptr(out), _stream(X0, out))
    _check(st, "ciq_mlp_features", allow=(CIQ_OK,))
    return out


def ciq_mlp_normaliser(F, Y, theta):
    st = lib().ciq_mlp_normaliser(_ptr(F), _ptr(Y), int(F.shape[0]), _ptr(theta), _stream(F, Y, theta))
    _check(st, "ciq_mlp_normaliser", allow=(CIQ_OK,))
    return theta


def ciq_mlp_init(theta, seed):
    st = lib().ciq_mlp_init(_ptr(theta), int(seed), _stream(theta))
    _check(st, "ciq_mlp_init", allow=(CIQ_OK,))
    return theta


def ciq_mlp_loss_grad(theta, F, Y, grad=None):
    """(loss, grad): full-batch loss and its gradient (float64 device tensor)."""
    import torch
    if grad is None:
        grad = torch.empty(CIQ_MLP_PARAMS, dtype=torch.float64, device=theta.device)
    loss = ctypes.c_double()
    st = lib().ciq_mlp_loss_grad(_ptr(theta), _ptr(F), _ptr(Y), int(F.shape[0]), ctypes.byref(loss), _ptr(grad),
                                 _stream(theta, F, Y, grad))
    _check(st, "ciq_mlp_loss_grad", allow=(CIQ_OK,))
    return loss.value, grad


def ciq_mlp_train(theta, adam, F, Y, steps, batch, lr, seed, first_step=1, losses=None):
    st = lib().ciq_mlp_train(_ptr(theta), _ptr(adam), _ptr(F), _ptr(Y), int(F.shape[0]), int(steps), int(batch),
                             float(lr), int(seed), int(first_step), _ptr(losses), _stream(theta, adam, F, Y))
    _check(st, "ciq_mlp_train", allow=(CIQ_OK,))
    return theta


def ciq_mlp_predict(theta, F, out=None, bf16=True):
    import torch
    if out is None:
        out = torch.empty((F.shape[0], CIQ_MLP_OUTPUTS), dtype=torch.float32, device=F.device)
    st = lib().ciq_mlp_predict(_ptr(theta), _ptr(F), int(F.shape[0]), _ptr(out), 1 if bf16 else 0,
                               _stream(theta, F, out))
    _check(st, "ciq_mlp_predict", allow=(CIQ_OK,))
    return out
