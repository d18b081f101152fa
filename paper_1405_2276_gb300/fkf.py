"""Python binding of the C-ABI in include/fkf.h (ctypes; argument marshalling only).

Every function here has the name of the C entry point it calls and performs
no arithmetic of the method: device work runs in libfkf.so.  Device buffers
are passed as torch CUDA tensors (their data_ptr()); host buffers as numpy
arrays.  A non-OK status raises FkfError carrying fkf_last_error().

The library is loaded from this package directory; importing this module on a
machine without the built library raises ImportError (there is no fallback).
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfkf.so")

FKF_OK, FKF_EINVAL, FKF_ENOMEM, FKF_ENOTSPD, FKF_ENOCONV, FKF_ETIMEOUT, FKF_ECUDA, FKF_ESTATE = range(8)
STATUS_NAMES = {
    0: "FKF_OK", 1: "FKF_EINVAL", 2: "FKF_ENOMEM", 3: "FKF_ENOTSPD",
    4: "FKF_ENOCONV", 5: "FKF_ETIMEOUT", 6: "FKF_ECUDA", 7: "FKF_ESTATE",
}
FKF_FP64, FKF_FP32 = 0, 1
FKF_STEP_INPUTS_ON_DEVICE = 1
FKF_STEP_SKIP_MEAN_SYNC = 2
FKF_STEP_FULL_UPDATE = 4
FKF_STEP_ALLOW_FIXED_H = 8
FKF_STEP_DENSE_HT = 16


class fkf_matern(C.Structure):
    _fields_ = [("nu", C.c_double), ("ell", C.c_double), ("sigma2", C.c_double)]


class fkf_hparams(C.Structure):
    _fields_ = [("leaf", C.c_int32), ("eta", C.c_double), ("aca_tol", C.c_double), ("k_cap", C.c_int32)]


class fkf_hmat_info(C.Structure):
    _fields_ = [
        ("n", C.c_int64), ("dim", C.c_int32), ("precision", C.c_int32),
        ("n_clusters", C.c_int64), ("n_leaves", C.c_int64), ("n_far", C.c_int64), ("n_near", C.c_int64),
        ("far_entries", C.c_int64), ("near_entries", C.c_int64), ("max_rank", C.c_int64),
        ("mean_rank", C.c_double), ("device_bytes", C.c_int64), ("flops_per_col", C.c_int64),
        ("bytes_per_col", C.c_int64), ("operator_bytes", C.c_int64), ("build_seconds", C.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class fkf_step_desc(C.Structure):
    _fields_ = [
        ("filter", C.c_void_p), ("y", C.c_void_p), ("m", C.c_int32), ("H_rowptr", C.c_void_p),
        ("H_col", C.c_void_p), ("H_val", C.c_void_p), ("R", C.c_void_p), ("r_scalar", C.c_double),
        ("nll", C.c_double), ("status", C.c_int32), ("merged", C.c_int32),
    ]


class fkf_filter_stats(C.Structure):
    _fields_ = [("k", C.c_int64), ("alpha", C.c_double), ("r", C.c_int32), ("last_path", C.c_int32),
                ("diagonal", C.c_int32), ("gep_rank", C.c_int32), ("new_dirs", C.c_int32), ("t_eig", C.c_int32),
                ("t_lmax", C.c_double), ("chol_exact_retries", C.c_int64)]


class FkfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built; run __graft_entry__.build() or paper_1405_2276_gb300/builder.py")
_lib = C.CDLL(LIB_PATH)

_P = C.c_void_p
_sigs = {
    "fkf_create": (C.c_int, [C.POINTER(_P), C.c_int32, _P]),
    "fkf_destroy": (None, [_P]),
    "fkf_last_error": (C.c_char_p, [_P]),
    "fkf_launch_count": (C.c_int64, [_P]),
    "fkf_library_call_count": (C.c_int64, [_P]),
    "fkf_hmatrix_build": (C.c_int, [_P, _P, C.c_int64, C.c_int32, fkf_matern, fkf_hparams, C.c_int, C.POINTER(_P)]),
    "fkf_hmatrix_info": (C.c_int, [_P, C.POINTER(fkf_hmat_info)]),
    "fkf_hmatrix_apply": (C.c_int, [_P, _P, C.c_int64, _P, C.c_int64, C.c_int64]),
    "fkf_hmatrix_apply_clustered": (C.c_int, [_P, _P, C.c_int64, _P, C.c_int64, C.c_int64]),
    "fkf_hmatrix_apply_adjoint": (C.c_int, [_P, _P, C.c_int64, _P, C.c_int64, _P, C.c_int64, C.c_int64,
                                            C.POINTER(C.c_double)]),
    "fkf_hmatrix_apply_clustered_noalloc": (C.c_int, [_P, _P, C.c_int64, _P, C.c_int64, C.c_int64]),
    "fkf_gemm_f64": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_int64, C.c_int64, C.c_int64, C.c_double, _P, C.c_int64,
                               _P, C.c_int64, C.c_double, _P, C.c_int64]),
    "fkf_rotate_f32": (C.c_int, [_P, _P, C.c_int64, C.c_int64, C.c_int32, _P, C.c_int64, C.c_int64, C.c_int32, _P,
                                 C.c_int64]),
    "fkf_hmatrix_permutation": (C.c_int, [_P, _P]),
    "fkf_hmatrix_densify": (C.c_int, [_P, _P]),
    "fkf_hmatrix_destroy": (None, [_P]),
    "fkf_filter_create": (C.c_int, [_P, _P, C.c_double, C.c_double, C.c_int32, C.c_int32, C.POINTER(_P)]),
    "fkf_filter_destroy": (None, [_P]),
    "fkf_filter_step": (C.c_int, [_P, _P, C.c_int32, _P, _P, _P, _P, C.c_double, C.c_int32, _P]),
    "fkf_filter_step_ekf": (C.c_int, [_P, _P, C.c_int32, _P, _P, _P, _P, C.c_double, C.c_double, C.c_int32, _P]),
    "fkf_filter_set_refresh": (C.c_int, [_P, C.c_int32]),
    "fkf_filter_set_randomized_ghep": (C.c_int, [_P, C.c_int32, C.c_int32, _P]),
    "fkf_filter_get": (C.c_int, [_P, _P, _P, _P, _P, _P, C.c_int64]),
    "fkf_variance": (C.c_int, [_P, _P]),
    "fkf_conditional_realization": (C.c_int, [_P, _P, C.c_int32, _P]),
    "fkf_uncertainty_scalars": (C.c_int, [_P, _P, _P]),
    "fkf_filter_orthonormality": (C.c_int, [_P, _P]),
    "fkf_filter_refresh": (C.c_int, [_P]),
    "fkf_filter_checkpoint": (C.c_int, [_P, C.c_char_p]),
    "fkf_filter_restore": (C.c_int, [_P, C.c_char_p]),
    "fkf_filter_phase_times": (C.c_int, [_P, _P]),
    "fkf_filter_set_tolerances": (C.c_int, [_P, C.c_double, C.c_double, C.c_double]),
    "fkf_nll_gradient": (C.c_int, [_P, C.c_int32, C.c_int32, _P, _P, _P, _P, C.c_double, _P, C.c_double,
                                   _P, _P, _P, _P, _P]),
    "fkf_filter_step_batched": (C.c_int, [C.POINTER(fkf_step_desc), C.c_int32, C.c_int32]),
    "fkf_filter_get_stats": (C.c_int, [_P, C.POINTER(fkf_filter_stats)]),
    "fkf_hmatrix_set_engine": (C.c_int, [_P, C.c_int32]),
    "fkf_hmatrix_set_wait_limit": (C.c_int, [_P, C.c_int64]),
    "fkf_eigh": (C.c_int, [_P, C.c_int32, _P, _P, C.c_int32]),
    "fkf_hmatrix_get_engine": (C.c_int, [_P, C.POINTER(C.c_int32)]),
    "fkf_hmatrix_release_values": (C.c_int, [_P]),
    "fkf_hmatrix_autotune": (C.c_int, [_P, C.c_int64, C.POINTER(C.c_int32), C.POINTER(C.c_double)]),
}
for _name, (_res, _args) in _sigs.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_sigs)


def _ptr(x):
    """Pointer of a torch tensor (data_ptr), numpy array, int or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    raise TypeError(type(x))


class Handle:
    """Opaque pointer with the context it reports errors on."""

    def __init__(self, ptr, ctx=None):
        self.ptr = ptr
        self.ctx = ctx if ctx is not None else self


def _check(status, ctx):
    if status != FKF_OK:
        msg = _lib.fkf_last_error(ctx.ptr if ctx is not None else None)
        raise FkfError(status, msg.decode() if msg else "")


# ---- context -----------------------------------------------------------------
def fkf_create(device: int = 0, cuda_stream: int | None = None) -> Handle:
    out = _P()
    st = _lib.fkf_create(C.byref(out), device, cuda_stream)
    if st != FKF_OK:
        raise FkfError(st, "fkf_create failed (no CUDA device or bad arguments)")
    return Handle(out.value)


def fkf_destroy(ctx: Handle) -> None:
    _lib.fkf_destroy(ctx.ptr)


def fkf_last_error(ctx: Handle) -> str:
    return _lib.fkf_last_error(ctx.ptr).decode()


def fkf_launch_count(ctx: Handle) -> int:
    return int(_lib.fkf_launch_count(ctx.ptr))


def fkf_library_call_count(ctx: Handle) -> int:
    return int(_lib.fkf_library_call_count(ctx.ptr))


# ---- H-matrix ------------------------------------------------------------------
def fkf_hmatrix_build(ctx, points, nu, ell, sigma2, leaf=64, eta=1.0, aca_tol=1e-8, k_cap=32, precision=FKF_FP64):
    pts = np.ascontiguousarray(points, dtype=np.float64)
    n, dim = pts.shape
    out = _P()
    st = _lib.fkf_hmatrix_build(ctx.ptr, pts.ctypes.data, n, dim, fkf_matern(nu, ell, sigma2),
                                fkf_hparams(leaf, eta, aca_tol, k_cap), precision, C.byref(out))
    _check(st, ctx)
    return Handle(out.value, ctx)


def fkf_hmatrix_info(h) -> dict:
    info = fkf_hmat_info()
    _check(_lib.fkf_hmatrix_info(h.ptr, C.byref(info)), h.ctx)
    return info.as_dict()


def fkf_hmatrix_apply(h, X, Y, ncols=None, ldx=None, ldy=None):
    ncols = X.shape[1] if ncols is None else ncols
    ldx = X.stride(0) if ldx is None else ldx
    ldy = Y.stride(0) if ldy is None else ldy
    _check(_lib.fkf_hmatrix_apply(h.ptr, _ptr(X), ldx, _ptr(Y), ldy, ncols), h.ctx)


def fkf_hmatrix_apply_adjoint(h, gY, Y, gX):
    """gX = Gamma_H gY; returns dL/dsigma2 = <gY, Y> / sigma2 (Y the forward result)."""
    ncols = gY.shape[1] if gY.dim() > 1 else 1
    g = C.c_double(0.0)
    _check(_lib.fkf_hmatrix_apply_adjoint(h.ptr, _ptr(gY), ncols, _ptr(Y), ncols, _ptr(gX), ncols, ncols,
                                          C.byref(g)), h.ctx)
    return g.value


def fkf_hmatrix_apply_clustered(h, X, Y, ncols=None, ldx=None, ldy=None):
    ncols = X.shape[1] if ncols is None else ncols
    ldx = X.stride(0) if ldx is None else ldx
    ldy = Y.stride(0) if ldy is None else ldy
    _check(_lib.fkf_hmatrix_apply_clustered(h.ptr, _ptr(X), ldx, _ptr(Y), ldy, ncols), h.ctx)


def fkf_hmatrix_apply_clustered_noalloc(h, X, Y, ncols=None, ldx=None, ldy=None):
    """Same product as fkf_hmatrix_apply_clustered, for callers that cannot
    allocate device memory: the library uses its fixed static scratch
    (FKF_NOALLOC_SCRATCH_BYTES per GPU) and never calls cudaMalloc."""
    ncols = X.shape[1] if ncols is None else ncols
    ldx = X.stride(0) if ldx is None else ldx
    ldy = Y.stride(0) if ldy is None else ldy
    _check(_lib.fkf_hmatrix_apply_clustered_noalloc(h.ptr, _ptr(X), ldx, _ptr(Y), ldy, ncols), h.ctx)


def fkf_rotate_f32(ctx, A, E, C, K=None, ncols=None):
    """C[:, :ncols] = A[:, :K] @ E[:K, :ncols] on the tensor cores (FP32
    row-major CUDA tensors, any leading dimensions)."""
    K = A.shape[1] if K is None else K
    ncols = C.shape[1] if ncols is None else ncols
    _check(_lib.fkf_rotate_f32(ctx.ptr, _ptr(A), A.stride(0), A.shape[0], K, _ptr(E), E.stride(0), E.shape[0], ncols,
                               _ptr(C), C.stride(0)), ctx)


def fkf_gemm_f64(ctx, A, B, C, alpha=1.0, beta=0.0, trans_a=False, trans_b=False):
    """C = alpha op(A) op(B) + beta C on the tensor cores (FP64 row-major CUDA
    tensors, any leading dimensions; FP64 products from integer slices)."""
    M, N = C.shape
    K = A.shape[0] if trans_a else A.shape[1]
    _check(_lib.fkf_gemm_f64(ctx.ptr, int(trans_a), int(trans_b), M, N, K, float(alpha), _ptr(A), A.stride(0),
                             _ptr(B), B.stride(0), float(beta), _ptr(C), C.stride(0)), ctx)


def fkf_hmatrix_set_engine(h, engine: int) -> None:
    """FP32 operators: 2 = tensor cores with scaled 2xFP16 (default), 1 = tensor
    cores with 3xTF32, 0 = SIMT tile engine.  FP64 operators: 0 = FP64 SIMT
    tile engine (default), 3 = tensor cores with 7-bit integer slices."""
    _check(_lib.fkf_hmatrix_set_engine(h.ptr, engine), h.ctx)


def fkf_hmatrix_autotune(h, ncols: int):
    """Pick the faster tensor-core pipeline shape for this operator; returns
    (variant, ms per apply of ncols columns)."""
    v = C.c_int32()
    ms = C.c_double()
    _check(_lib.fkf_hmatrix_autotune(h.ptr, ncols, C.byref(v), C.byref(ms)), h.ctx)
    return v.value, ms.value


def fkf_eigh(ctx, A, w, want=None) -> None:
    """Symmetric eigendecomposition on the device: A (n x n torch CUDA float64,
    overwritten: rows 0..want-1 = eigenvectors of the want largest eigenvalues,
    ascending), w (n, float64): all eigenvalues ascending."""
    n = A.shape[0]
    want = n if want is None else int(want)
    _check(_lib.fkf_eigh(ctx.ptr, n, _ptr(A), _ptr(w), want), ctx)


def fkf_hmatrix_set_wait_limit(h, polls: int) -> None:
    _check(_lib.fkf_hmatrix_set_wait_limit(h.ptr, int(polls)), h.ctx)


def fkf_hmatrix_release_values(h) -> None:
    """Free the FP32 operator's device value copies (keeps the tensor-core stream)."""
    _check(_lib.fkf_hmatrix_release_values(h.ptr), h.ctx)


def fkf_hmatrix_get_engine(h) -> int:
    e = C.c_int32()
    _check(_lib.fkf_hmatrix_get_engine(h.ptr, C.byref(e)), h.ctx)
    return e.value


def fkf_hmatrix_permutation(h, n):
    out = np.zeros(n, dtype=np.int64)
    _check(_lib.fkf_hmatrix_permutation(h.ptr, out.ctypes.data), h.ctx)
    return out


def fkf_hmatrix_densify(h, n):
    out = np.zeros((n, n))
    _check(_lib.fkf_hmatrix_densify(h.ptr, out.ctypes.data), h.ctx)
    return out


def fkf_hmatrix_destroy(h) -> None:
    _lib.fkf_hmatrix_destroy(h.ptr)


# ---- filter --------------------------------------------------------------------
def fkf_filter_create(h, s0=None, alpha0=0.0, trunc_tol=1e-12, m_max=1024, r_max=2048):
    s0p = None
    if s0 is not None:
        s0 = np.ascontiguousarray(s0, dtype=np.float64)
        s0p = s0.ctypes.data
    out = _P()
    _check(_lib.fkf_filter_create(h.ptr, s0p, alpha0, trunc_tol, m_max, r_max, C.byref(out)), h.ctx)
    return Handle(out.value, h.ctx)


def fkf_filter_destroy(f) -> None:
    _lib.fkf_filter_destroy(f.ptr)


def fkf_filter_step(f, y, m, rowptr, col, val, R=None, r_scalar=0.0, flags=0, want_nll=True):
    """y, rowptr (int64), col (int32), val (float64), R: numpy host arrays or,
    with FKF_STEP_INPUTS_ON_DEVICE in flags, torch CUDA tensors."""
    nll = C.c_double(0.0)
    st = _lib.fkf_filter_step(f.ptr, _ptr(y), m, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(R), r_scalar, flags,
                              C.byref(nll) if want_nll else None)
    _check(st, f.ctx)
    return nll.value


def fkf_filter_step_ekf(f, y, m, rowptr, col, val, boxcox_a, R=None, r_scalar=0.0, flags=0, want_nll=True):
    """Extended filter step with the Box-Cox map s(x) = ((x + a)/a)^a:
    y = H s(x) + v; arguments as fkf_filter_step plus a = boxcox_a."""
    nll = C.c_double(0.0)
    st = _lib.fkf_filter_step_ekf(f.ptr, _ptr(y), m, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(R), r_scalar,
                                  float(boxcox_a), flags, C.byref(nll) if want_nll else None)
    _check(st, f.ctx)
    return nll.value


def fkf_filter_step_batched(entries, flags=0, return_merged=False):
    """entries: list of (filter, y, rowptr, col, val, R or None, r_scalar), each
    filter on its own context.  Returns the list of per-filter NLLs (and, with
    return_merged, whether each step's H-apply ran in the merged launches);
    raises FkfError (with the first failing status) if any step failed."""
    nb = len(entries)
    descs = (fkf_step_desc * nb)()
    keep = []
    for i, (f, y, rowptr, col, val, R, rs) in enumerate(entries):
        y = np.ascontiguousarray(y, dtype=np.float64) if isinstance(y, np.ndarray) else y
        keep.append(y)
        d = descs[i]
        d.filter = f.ptr
        d.y = _ptr(y)
        d.m = int(rowptr.shape[0] - 1)
        d.H_rowptr, d.H_col, d.H_val = _ptr(rowptr), _ptr(col), _ptr(val)
        d.R = _ptr(R)
        d.r_scalar = rs
    st = _lib.fkf_filter_step_batched(descs, nb, flags)
    if st != FKF_OK:
        bad = next(i for i in range(nb) if descs[i].status != FKF_OK) if any(
            descs[i].status != FKF_OK for i in range(nb)) else 0
        _check(st, entries[bad][0].ctx)
    nlls = [descs[i].nll for i in range(nb)]
    if return_merged:
        return nlls, [bool(descs[i].merged) for i in range(nb)]
    return nlls


def fkf_filter_get(f, n, want_s=True, want_D=True, W=None):
    alpha = C.c_double(0)
    r = C.c_int32(0)
    s = np.zeros(n) if want_s else None
    # rank first, to size D
    _check(_lib.fkf_filter_get(f.ptr, None, C.byref(alpha), C.byref(r), None, None, 0), f.ctx)
    D = np.zeros(max(r.value, 1)) if want_D else None
    _check(_lib.fkf_filter_get(f.ptr, _ptr(s), None, None, _ptr(D), _ptr(W), W.stride(0) if W is not None else 0),
           f.ctx)
    return dict(s=s, alpha=alpha.value, r=r.value, D=D[: r.value] if D is not None else None)


def fkf_filter_get_stats(f) -> dict:
    s = fkf_filter_stats()
    _check(_lib.fkf_filter_get_stats(f.ptr, C.byref(s)), f.ctx)
    return {k: getattr(s, k) for k, _ in s._fields_}


def fkf_variance(f, var_dev) -> None:
    _check(_lib.fkf_variance(f.ptr, _ptr(var_dev)), f.ctx)


def fkf_conditional_realization(f, a_dev, out_dev, ns=None) -> None:
    ns = a_dev.shape[1] if ns is None else ns
    _check(_lib.fkf_conditional_realization(f.ptr, _ptr(a_dev), ns, _ptr(out_dev)), f.ctx)


def fkf_uncertainty_scalars(f):
    e = C.c_double(0)
    t = C.c_double(0)
    _check(_lib.fkf_uncertainty_scalars(f.ptr, C.byref(e), C.byref(t)), f.ctx)
    return e.value, t.value


def fkf_filter_orthonormality(f) -> float:
    e = C.c_double(0)
    _check(_lib.fkf_filter_orthonormality(f.ptr, C.byref(e)), f.ctx)
    return e.value


def fkf_filter_refresh(f) -> None:
    _check(_lib.fkf_filter_refresh(f.ptr), f.ctx)


def fkf_filter_set_randomized_ghep(f, k: int, p: int = 0, omega=None) -> None:
    """k modes from a sketch of k + p Gaussian columns omega (torch CUDA float64,
    N x (k + p), original point order); k = 0: the exact GEP."""
    _check(_lib.fkf_filter_set_randomized_ghep(f.ptr, int(k), int(p), _ptr(omega)), f.ctx)


def fkf_filter_set_refresh(f, every: int) -> None:
    _check(_lib.fkf_filter_set_refresh(f.ptr, int(every)), f.ctx)


def fkf_filter_checkpoint(f, path: str) -> None:
    _check(_lib.fkf_filter_checkpoint(f.ptr, path.encode()), f.ctx)


def fkf_filter_restore(f, path: str) -> None:
    _check(_lib.fkf_filter_restore(f.ptr, path.encode()), f.ctx)


def fkf_nll_gradient(h, y, rowptr, col, val, rho, s0=None, alpha0=0.0, want_grads=True):
    """Summed NLL of K fixed-H steps and its gradients (host numpy arrays).
    y: (K, m).  Returns (nll, grad_y (K, m), grad_s0 (N,), grad_sigma2, grad_rho)."""
    y = np.ascontiguousarray(y, dtype=np.float64)
    K, m = y.shape
    n = fkf_hmatrix_info(h)["n"]
    nll = C.c_double(0)
    gy = np.zeros((K, m)) if want_grads else None
    gs = np.zeros(n) if want_grads else None
    gsig = C.c_double(0)
    grho = C.c_double(0)
    s0p = None
    if s0 is not None:
        s0 = np.ascontiguousarray(s0, dtype=np.float64)
        s0p = s0.ctypes.data
    st = _lib.fkf_nll_gradient(h.ptr, K, m, y.ctypes.data, _ptr(rowptr), _ptr(col), _ptr(val), rho, s0p, alpha0,
                               C.byref(nll), _ptr(gy), _ptr(gs), C.byref(gsig) if want_grads else None,
                               C.byref(grho) if want_grads else None)
    _check(st, h.ctx)
    return nll.value, gy, gs, gsig.value, grho.value


def fkf_filter_set_tolerances(f, gep_tol, orth_tol, trunc_tol) -> None:
    _check(_lib.fkf_filter_set_tolerances(f.ptr, gep_tol, orth_tol, trunc_tol), f.ctx)


def fkf_filter_phase_times(f):
    out = (C.c_double * 6)()
    _check(_lib.fkf_filter_phase_times(f.ptr, out), f.ctx)
    return list(out)
