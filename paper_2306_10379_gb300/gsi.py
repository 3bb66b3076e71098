"""Python binding of libgsi.so (ctypes). Argument marshalling only: every step
of the method runs in the library's CUDA kernels. PyTorch supplies device
memory and the current stream.

If libgsi.so has not been built this module raises on first use; there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgsi.so")

GSI_OK, GSI_ERR_ARG, GSI_ERR_CUDA, GSI_ERR_OOM, GSI_ERR_NOCONV, GSI_ERR_BREAKDOWN, \
    GSI_ERR_NONFINITE, GSI_ERR_TIMEOUT = range(8)
GSI_CSR, GSI_SELL, GSI_DENSE = 0, 1, 2
GSI_SD, GSI_CG, GSI_CHEB, GSI_LOBCG = 0, 1, 2, 3
GSI_PREC_DF64, GSI_PREC_F64, GSI_PREC_MIXED = 0, 1, 2
PRECISIONS = {"df64": GSI_PREC_DF64, "f64": GSI_PREC_F64, "mixed": GSI_PREC_MIXED}
KERNEL_CLASSES = ["spmm", "gram", "blockmul", "small", "reduce"]

EXPORTED = [
    "gsi_default_opts", "gsi_create", "gsi_step", "gsi_solve", "gsi_get_basis", "gsi_state_ptrs",
    "gsi_destroy", "gsi_status_str", "gsi_last_error", "gsi_spmm_csr", "gsi_sell_size",
    "gsi_csr_to_sell", "gsi_spmm_sell", "gsi_gram", "gsi_residual", "gsi_linesearch",
    "gsi_retract", "gsi_df_spmm_csr", "gsi_oz_gemm", "gsi_oz_gram", "gsi_reset",
    "gsi_profile_enable", "gsi_profile_read", "gsi_launch_count", "gsi_oz_dense_apply",
    "gsi_oz_gram_noalloc", "gsi_measure_fma_peaks", "gsi_set_operator", "gsi_set_wait_limit",
    "gsi_device_timeouts", "gsi_create_hermitian", "gsi_get_basis_hermitian", "gsi_csr_to_dia",
    "gsi_df_spmm_dia",
]


class GsiError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = _lib().gsi_status_str(status).decode()
        extra = _lib().gsi_last_error().decode()
        super().__init__(f"{where}: {msg}" + (f" ({extra})" if extra and status == GSI_ERR_CUDA else ""))


class Matrix(ctypes.Structure):
    _fields_ = [("fmt", ctypes.c_int32), ("n", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("rowptr", ctypes.c_void_p), ("colidx", ctypes.c_void_p), ("val", ctypes.c_void_p),
                ("sell_C", ctypes.c_int32), ("sell_sigma", ctypes.c_int32),
                ("on_device", ctypes.c_int32)]


class ZMatrix(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("rowptr", ctypes.c_void_p),
                ("colidx", ctypes.c_void_p), ("val", ctypes.c_void_p), ("on_device", ctypes.c_int32)]


class Opts(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int32), ("which", ctypes.c_int32), ("tol", ctypes.c_double),
                ("anorm", ctypes.c_double), ("max_iters", ctypes.c_int32),
                ("k_restart", ctypes.c_int32), ("recompute_every", ctypes.c_int32),
                ("explicit_ax", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("cheb_degree", ctypes.c_int32), ("cheb_lo", ctypes.c_double),
                ("cheb_hi", ctypes.c_double), ("cheb_scale", ctypes.c_double),
                ("mixed_switch", ctypes.c_double), ("stop_rule", ctypes.c_int32),
                ("cheb_adaptive", ctypes.c_int32), ("cheb_guard", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("matvecs", ctypes.c_int32),
                ("restarts", ctypes.c_int32), ("brent_evals", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("rel_residual", ctypes.c_double),
                ("rel_residual_inf", ctypes.c_double), ("trace", ctypes.c_double),
                ("last_step", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2306_10379_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        sig = {
            "gsi_default_opts": [ctypes.POINTER(Opts)],
            "gsi_create": [ctypes.POINTER(Matrix), i32, vp, i32, ctypes.POINTER(Opts), vp,
                           ctypes.POINTER(vp)],
            "gsi_step": [vp, i32, ctypes.POINTER(Info)],
            "gsi_solve": [vp, ctypes.POINTER(Info)],
            "gsi_get_basis": [vp, vp, vp, i32],
            "gsi_state_ptrs": [vp, ctypes.POINTER(vp), ctypes.POINTER(vp)],
            "gsi_destroy": [vp],
            "gsi_spmm_csr": [i64, vp, vp, vp, i32, vp, vp, vp],
            "gsi_sell_size": [i64, vp, i32, i32, ctypes.POINTER(i64), ctypes.POINTER(i64)],
            "gsi_csr_to_sell": [i64, vp, vp, vp, i32, i32, vp, vp, vp, vp, vp],
            "gsi_spmm_sell": [i64, i64, i32, vp, vp, vp, vp, vp, i32, vp, vp, vp],
            "gsi_gram": [i64, i32, i32, vp, vp, vp, vp],
            "gsi_residual": [i64, i32, vp, vp, vp, vp, vp],
            "gsi_linesearch": [i32, vp, vp, vp, vp, vp, vp, vp, vp, i32, vp],
            "gsi_retract": [i64, i32, dbl, vp, vp, vp, vp, vp, vp],
            "gsi_df_spmm_csr": [i64, vp, vp, vp, i32, vp, vp, vp],
            "gsi_oz_gemm": [i64, i32, i32, vp, vp, vp, vp, dbl, dbl, i32, vp, vp, vp, vp, vp],
            "gsi_oz_gram": [i64, i32, i32, vp, vp, i32, vp, vp],
            "gsi_oz_dense_apply": [i64, i32, vp, vp, vp, i32, vp],
            "gsi_reset": [vp, vp, i32],
            "gsi_batched_plan": [i32, vp, vp, vp, i32, i32, vp, ctypes.POINTER(i32), vp, vp, vp, i32],
            "gsi_batched_create": [i32, vp, vp, vp, vp, vp, vp, vp, ctypes.POINTER(Opts), vp,
                                   ctypes.POINTER(vp)],
            "gsi_batched_set_tiles": [vp, i32, i32, i32],
            "gsi_batched_get_tiles": [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                      ctypes.POINTER(i32)],
            "gsi_batched_last_plan": [vp, ctypes.POINTER(i32), vp, vp, vp, i32],
            "gsi_batched_tune": [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                 ctypes.POINTER(dbl)],
            "gsi_batched_reset": [vp],
            "gsi_batched_step": [vp, i32],
            "gsi_batched_solve": [vp, i32, ctypes.POINTER(i32)],
            "gsi_batched_info": [vp, i32, ctypes.POINTER(Info), ctypes.POINTER(i32)],
            "gsi_batched_get_basis": [vp, i32, vp, vp],
            "gsi_batched_destroy": [vp],
            "gsi_batched_restart": [vp, vp, i32],
            "gsi_mlp_create": [i32, i32, i32, i32, vp, vp, ctypes.POINTER(vp)],
            "gsi_mlp_get_params": [vp, vp, vp],
            "gsi_mlp_forward": [vp, i32, vp, vp],
            "gsi_mlp_backward": [vp, i32, vp, vp],
            "gsi_mlp_adam": [vp, dbl, dbl, dbl, dbl],
            "gsi_mlp_destroy": [vp],
            "gsi_warm_loss_grad": [i32, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, ctypes.c_float, vp],
            "gsi_warm_train_step": [vp, i32, vp, i32, i32, vp, vp, vp, vp, dbl, ctypes.POINTER(dbl)],
            "gsi_prolong": [i32, i32, i32, i32, vp, vp, vp],
            "gsi_restrict": [i32, i32, i32, i32, vp, vp, vp],
            "gsi_gemm_bf16": [i32, i32, i32, vp, i64, i64, vp, i64, i64, vp, i64, ctypes.c_float,
                              ctypes.c_float, vp, vp, i32, vp],
            "gsi_set_wait_limit": [i32],
            "gsi_csr_to_dia": [i64, vp, vp, vp, i32, ctypes.POINTER(i32), vp, vp],
            "gsi_df_spmm_dia": [i64, i32, vp, vp, i32, vp, vp, vp],
            "gsi_set_operator": [vp, ctypes.POINTER(Matrix), dbl],
            "gsi_create_hermitian": [ctypes.POINTER(ZMatrix), i32, vp, i32, ctypes.POINTER(Opts), vp,
                                     ctypes.POINTER(vp)],
            "gsi_get_basis_hermitian": [vp, vp, vp, i32],
            "gsi_device_timeouts": [ctypes.POINTER(i64)],
            "gsi_profile_enable": [vp, i32],
            "gsi_profile_read": [vp, i32, ctypes.POINTER(i64), ctypes.POINTER(dbl),
                                 ctypes.POINTER(dbl), ctypes.POINTER(dbl)],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.gsi_status_str.argtypes = [ctypes.c_int]
        L.gsi_status_str.restype = ctypes.c_char_p
        L.gsi_last_error.argtypes = []
        L.gsi_last_error.restype = ctypes.c_char_p
        L.gsi_launch_count.argtypes = []
        L.gsi_launch_count.restype = ctypes.c_int64
        L.gsi_set_tensor_path.argtypes = [i32]
        L.gsi_set_tensor_path.restype = ctypes.c_int
        L.gsi_tensor_path.argtypes = []
        L.gsi_tensor_path.restype = ctypes.c_int32
        L.gsi_measure_fma_peaks.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        L.gsi_measure_fma_peaks.restype = ctypes.c_int
        L.gsi_mlp_num_params.argtypes = [i32, i32, i32]
        L.gsi_mlp_num_params.restype = ctypes.c_int64
        _LIB = L
    return _LIB


def lib():
    """The loaded ctypes library (raises if libgsi.so is missing)."""
    return _lib()


def _check(status, where):
    if status != GSI_OK:
        raise GsiError(status, where)


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t, dtype=None, shape=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected dtype {dtype}, got {t.dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


class _DeviceArray:
    """Zero-copy view of library-owned device memory via __cuda_array_interface__."""

    def __init__(self, ptr, shape, typestr="<f8"):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}


# ----------------------------------------------------------------------------
# Kernel-level entry points (torch CUDA tensors in, results written in place)
# ----------------------------------------------------------------------------

def spmm_csr(rowptr, colidx, val, X, W, stream=None):
    import torch
    n, p = X.shape
    _check(lib().gsi_spmm_csr(n, _dptr(rowptr, torch.int64), _dptr(colidx, torch.int32),
                              _dptr(val, torch.float64), p, _dptr(X, torch.float64),
                              _dptr(W, torch.float64, (n, p)), _stream(stream)), "gsi_spmm_csr")


def csr_to_sell(n, rowptr, colidx, val, C=32, sigma=32):
    """Host conversion (numpy arrays in, numpy arrays out)."""
    rowptr = np.ascontiguousarray(rowptr, np.int64)
    colidx = np.ascontiguousarray(colidx, np.int32)
    val = np.ascontiguousarray(val, np.float64)
    nch, tot = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().gsi_sell_size(n, rowptr.ctypes.data, C, sigma, ctypes.byref(nch), ctypes.byref(tot)),
           "gsi_sell_size")
    perm = np.empty(nch.value * C, np.int64)
    cptr = np.empty(nch.value + 1, np.int64)
    clen = np.empty(nch.value, np.int64)
    scol = np.empty(tot.value, np.int32)
    sval = np.empty(tot.value, np.float64)
    _check(lib().gsi_csr_to_sell(n, rowptr.ctypes.data, colidx.ctypes.data, val.ctypes.data, C, sigma,
                                 perm.ctypes.data, cptr.ctypes.data, clen.ctypes.data,
                                 scol.ctypes.data, sval.ctypes.data), "gsi_csr_to_sell")
    return perm, cptr, clen, scol, sval


def spmm_sell(n, C, perm, chunk_ptr, chunk_len, scol, sval, X, W, stream=None):
    import torch
    p = X.shape[1]
    nchunks = chunk_len.shape[0]
    _check(lib().gsi_spmm_sell(n, nchunks, C, _dptr(perm, torch.int64), _dptr(chunk_ptr, torch.int64),
                               _dptr(chunk_len, torch.int64), _dptr(scol, torch.int32),
                               _dptr(sval, torch.float64), p, _dptr(X, torch.float64),
                               _dptr(W, torch.float64, (n, p)), _stream(stream)), "gsi_spmm_sell")


def gram(U, V, G, stream=None):
    import torch
    n, p = U.shape
    q = V.shape[1]
    _check(lib().gsi_gram(n, p, q, _dptr(U, torch.float64), _dptr(V, torch.float64, (n, q)),
                          _dptr(G, torch.float64, (p, q)), _stream(stream)), "gsi_gram")


def residual(X, Y, C, R, stream=None):
    import torch
    n, p = X.shape
    _check(lib().gsi_residual(n, p, _dptr(X, torch.float64), _dptr(Y, torch.float64, (n, p)),
                              _dptr(C, torch.float64, (p, p)), _dptr(R, torch.float64, (n, p)),
                              _stream(stream)), "gsi_residual")


def linesearch(C, B, Gam, Z, XX, XD, M, out, precision="df64", stream=None):
    import torch
    p = C.shape[0]
    f = torch.float64
    pr = GSI_PREC_DF64 if precision == "df64" else GSI_PREC_F64
    _check(lib().gsi_linesearch(p, _dptr(C, f, (p, p)), _dptr(B, f, (p, p)), _dptr(Gam, f, (p, p)),
                                _dptr(Z, f, (p, p)), _dptr(XX, f, (p, p)), _dptr(XD, f, (p, p)),
                                _dptr(M, f, (p, p)), _dptr(out, f), pr, _stream(stream)),
           "gsi_linesearch")


def retract(t, M, X, D, Y, W, stream=None):
    import torch
    n, p = X.shape
    f = torch.float64
    _check(lib().gsi_retract(n, p, float(t), _dptr(M, f, (p, p)), _dptr(X, f), _dptr(D, f, (n, p)),
                             _dptr(Y, f, (n, p)), _dptr(W, f, (n, p)), _stream(stream)), "gsi_retract")


def set_tensor_path(path):
    """0 (default) and 2: tcgen05 kernels wherever they apply (p, q <= 64); 1: mma.sync only."""
    _check(lib().gsi_set_tensor_path(int(path)), "gsi_set_tensor_path")


def tensor_path():
    return int(lib().gsi_tensor_path())


def measure_fma_peaks(stream=None):
    """Measured float64 and float32 multiply-add throughput of the current GPU (TFLOP/s)."""
    out = np.zeros(2, np.float64)
    _check(lib().gsi_measure_fma_peaks(ctypes.c_void_p(out.ctypes.data), _stream(stream)),
           "gsi_measure_fma_peaks")
    return {"fp64_fma_tflops": float(out[0]), "fp32_fma_tflops": float(out[1])}


def set_wait_limit(polls):
    """Polls allowed to each bounded wait of the tensor-core kernels on the
    current device (negative: the default 2^24)."""
    _check(lib().gsi_set_wait_limit(int(polls)), "gsi_set_wait_limit")


def device_timeouts():
    """Bounded waits that ran out on the current device since the library was loaded."""
    c = ctypes.c_int64()
    _check(lib().gsi_device_timeouts(ctypes.byref(c)), "gsi_device_timeouts")
    return int(c.value)


def launch_count():
    """Kernels launched by libgsi in this process."""
    return int(lib().gsi_launch_count())


# ----------------------------------------------------------------------------
# df64 kernels: a df64 tensor is float32 with a trailing dimension of 2 (hi, lo)
# ----------------------------------------------------------------------------

def to_df(x):
    """float64 numpy array -> float32 array with trailing (hi, lo) axis."""
    x = np.asarray(x, dtype=np.float64)
    h = x.astype(np.float32)
    l = (x - h.astype(np.float64)).astype(np.float32)
    return np.stack([h, l], axis=-1)


def from_df(d):
    d = np.asarray(d)
    return d[..., 0].astype(np.float64) + d[..., 1].astype(np.float64)


def df_spmm_csr(rowptr, colidx, val_df, X_df, W_df, stream=None):
    import torch
    n, p = X_df.shape[0], X_df.shape[1]
    f = torch.float32
    _check(lib().gsi_df_spmm_csr(n, _dptr(rowptr, torch.int64), _dptr(colidx, torch.int32),
                                 _dptr(val_df, f), p, _dptr(X_df, f), _dptr(W_df, f, (n, p, 2)),
                                 _stream(stream)), "gsi_df_spmm_csr")


def csr_to_dia(n, rowptr, colidx, val, max_diags=8):
    """Host diagonal layout: (offsets int64, dia n x ndiag float64), or None
    when the nonzeros lie on more than max_diags diagonals."""
    rowptr = np.ascontiguousarray(rowptr, np.int64)
    colidx = np.ascontiguousarray(colidx, np.int32)
    val = np.ascontiguousarray(val, np.float64)
    nd = ctypes.c_int32()
    _check(lib().gsi_csr_to_dia(n, rowptr.ctypes.data, colidx.ctypes.data, None, max_diags, ctypes.byref(nd),
                                None, None), "gsi_csr_to_dia")
    if nd.value == 0:
        return None
    off = np.empty(nd.value, np.int64)
    dia = np.empty((n, nd.value), np.float64)
    _check(lib().gsi_csr_to_dia(n, rowptr.ctypes.data, colidx.ctypes.data, val.ctypes.data, max_diags,
                                ctypes.byref(nd), off.ctypes.data, dia.ctypes.data), "gsi_csr_to_dia")
    return off, dia


def df_spmm_dia(offsets, dia_df, X_df, W_df, stream=None):
    """W = A X for the diagonal layout (offsets host int64, dia_df a device df64
    tensor n x ndiag x 2)."""
    import torch
    n, p = X_df.shape[0], X_df.shape[1]
    off = np.ascontiguousarray(offsets, np.int64)
    f = torch.float32
    _check(lib().gsi_df_spmm_dia(n, int(off.size), ctypes.c_void_p(off.ctypes.data), _dptr(dia_df, f), p,
                                 _dptr(X_df, f), _dptr(W_df, f, (n, p, 2)), _stream(stream)), "gsi_df_spmm_dia")


def oz_gemm(U0, M0, out, s0=1.0, U1=None, M1=None, s1=0.0, E=(), c=(), stream=None):
    import torch
    n, p = U0.shape[0], U0.shape[1]
    f, d = torch.float32, torch.float64
    nk = 2 if U1 is not None else 1
    cc = np.zeros(4, np.float32)  # host memory: the scalars are read by the host
    for m, cm in enumerate(c):
        cc[2 * m:2 * m + 2] = to_df(np.float64(cm))
    E = list(E) + [None] * (2 - len(E))
    _check(lib().gsi_oz_gemm(n, p, nk, _dptr(U0, f), _dptr(U1, f) if U1 is not None else None,
                             _dptr(M0, d, (p, p)), _dptr(M1, d, (p, p)) if M1 is not None else None,
                             float(s0), float(s1), len([e for e in E if e is not None]),
                             _dptr(E[0], f) if E[0] is not None else None,
                             _dptr(E[1], f) if E[1] is not None else None,
                             ctypes.c_void_p(cc.ctypes.data),
                             _dptr(out, f, (n, p, 2)), _stream(stream)), "gsi_oz_gemm")


def oz_dense_apply(A_df, X_df, W_df, nd=7, stream=None):
    """W = A X for symmetric dense A (df64 tensors: A (n, n, 2), X, W (n, p, 2))."""
    import torch
    n, p = X_df.shape[0], X_df.shape[1]
    f = torch.float32
    _check(lib().gsi_oz_dense_apply(n, p, _dptr(A_df, f, (n, n, 2)), _dptr(X_df, f), _dptr(W_df, f, (n, p, 2)),
                                    int(nd), _stream(stream)), "gsi_oz_dense_apply")


def oz_gram(U, V, G, sym=False, stream=None):
    import torch
    n, p = U.shape[0], U.shape[1]
    q = V.shape[1]
    f = torch.float32
    _check(lib().gsi_oz_gram(n, p, q, _dptr(U, f), _dptr(V, f), 1 if sym else 0,
                             _dptr(G, torch.float64, (p, q)), _stream(stream)), "gsi_oz_gram")


# ----------------------------------------------------------------------------
# Solver context
# ----------------------------------------------------------------------------

class Dense:
    """A dense symmetric operator for Solver (val: n x n float64, numpy or CUDA tensor)."""

    dense = True

    def __init__(self, val):
        self.val = val
        self.n = int(val.shape[0])


class HermitianSolver:
    """gsi_create_hermitian / gsi_step / gsi_solve / gsi_get_basis_hermitian /
    gsi_destroy for a complex Hermitian A (object with n, rowptr, colidx and
    complex val, host numpy arrays) and a complex n x p start block."""

    def __init__(self, A, p, X0, method="cg", which=1, tol=1e-8, anorm=0.0, max_iters=10000,
                 precision="df64", stream=None):
        L = lib()
        rp = np.ascontiguousarray(A.rowptr, np.int64)
        ci = np.ascontiguousarray(A.colidx, np.int32)
        va = np.ascontiguousarray(np.asarray(A.val, np.complex128).view(np.float64))
        x0 = np.ascontiguousarray(np.asarray(X0, np.complex128).view(np.float64))
        self._keep = [rp, ci, va, x0]
        m = ZMatrix(int(A.n), int(ci.size), rp.ctypes.data, ci.ctypes.data, va.ctypes.data, 0)
        o = Opts()
        L.gsi_default_opts(ctypes.byref(o))
        o.method = {"sd": GSI_SD, "cg": GSI_CG}[method]
        o.which = int(which)
        o.tol = float(tol)
        o.anorm = float(anorm)
        o.max_iters = int(max_iters)
        o.precision = PRECISIONS[precision]
        self.n, self.p = int(A.n), int(p)
        ctx = ctypes.c_void_p()
        _check(L.gsi_create_hermitian(ctypes.byref(m), int(p), ctypes.c_void_p(x0.ctypes.data), 0, ctypes.byref(o),
                                      _stream(stream), ctypes.byref(ctx)), "gsi_create_hermitian")
        self._ctx = ctx

    def step(self, nsteps=1):
        info = Info()
        _check(lib().gsi_step(self._ctx, int(nsteps), ctypes.byref(info)), "gsi_step")
        return info.as_dict()

    def solve(self):
        info = Info()
        s = lib().gsi_solve(self._ctx, ctypes.byref(info))
        if s not in (GSI_OK, GSI_ERR_NOCONV):
            raise GsiError(s, "gsi_solve")
        return info.as_dict()

    def basis(self, evals=True):
        """(X, evals): the current complex iterate (n x p, orthonormal) and, with
        evals, its p Ritz values."""
        X = np.empty((self.n, self.p), np.complex128)
        ev = np.empty(self.p) if evals else None
        _check(lib().gsi_get_basis_hermitian(self._ctx, ctypes.c_void_p(X.ctypes.data),
                                             ctypes.c_void_p(ev.ctypes.data) if evals else None, 0),
               "gsi_get_basis_hermitian")
        return X, ev

    def close(self):
        if self._ctx:
            lib().gsi_destroy(self._ctx)
            self._ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _matrix(A, fmt, keep):
    """gsi_matrix for A (object with n, rowptr, colidx, val as numpy host arrays
    or torch CUDA tensors; or gsi.Dense); host arrays are kept alive in keep."""
    import torch
    dense = getattr(A, "dense", False)
    on_dev = isinstance(A.val, torch.Tensor)
    if dense:
        if on_dev:
            va = _dptr(A.val, torch.float64, (A.n, A.n))
        else:
            arr = np.ascontiguousarray(A.val, np.float64)
            keep.append(arr)
            va = ctypes.c_void_p(arr.ctypes.data)
        rp = ci = None
        nnz = 0
    elif on_dev:
        rp, ci, va = _dptr(A.rowptr, torch.int64), _dptr(A.colidx, torch.int32), _dptr(A.val, torch.float64)
        nnz = int(A.colidx.numel())
    else:
        arrs = [np.ascontiguousarray(A.rowptr, np.int64), np.ascontiguousarray(A.colidx, np.int32),
                np.ascontiguousarray(A.val, np.float64)]
        keep += arrs
        rp, ci, va = (ctypes.c_void_p(a.ctypes.data) for a in arrs)
        nnz = int(arrs[1].size)
    fm = GSI_DENSE if dense else (GSI_SELL if fmt == "sell" else GSI_CSR)
    return Matrix(fm, int(A.n), nnz, rp, ci, va, 32, 32, 1 if on_dev else 0)


class Solver:
    """gsi_create / gsi_step / gsi_solve / gsi_get_basis / gsi_destroy.

    A: object with n, rowptr, colidx, val (numpy host arrays or torch CUDA
    tensors). X0: n x p start block (numpy or torch CUDA float64)."""

    def __init__(self, A, p, X0, method="sd", which=1, tol=1e-8, anorm=0.0, max_iters=10000,
                 k_restart=0, recompute_every=50, explicit_ax=False, fmt="csr", precision="df64",
                 cheb_degree=8, cheb_interval=(0.0, 0.0), cheb_scale=0.0, mixed_switch=1e-5,
                 stop_rule="fro", cheb_adaptive=False, cheb_guard=0, stream=None):
        import torch
        L = lib()
        self._keep = []
        self._fmt = fmt
        m = _matrix(A, fmt, self._keep)
        o = Opts()
        L.gsi_default_opts(ctypes.byref(o))
        o.method = {"sd": GSI_SD, "cg": GSI_CG, "cheb": GSI_CHEB, "lobcg": GSI_LOBCG}[method]
        o.cheb_degree = int(cheb_degree)
        o.cheb_lo, o.cheb_hi = float(cheb_interval[0]), float(cheb_interval[1])
        o.cheb_scale = float(cheb_scale)
        o.which = int(which)
        o.tol = float(tol)
        o.anorm = float(anorm)
        o.max_iters = int(max_iters)
        o.k_restart = int(k_restart)
        o.recompute_every = int(recompute_every)
        o.explicit_ax = 1 if explicit_ax else 0
        if precision not in PRECISIONS:
            raise ValueError("precision must be one of " + ", ".join(PRECISIONS))
        o.precision = PRECISIONS[precision]
        o.mixed_switch = float(mixed_switch)
        o.stop_rule = {"fro": 0, "inf": 1}[stop_rule]
        o.cheb_adaptive = 1 if cheb_adaptive else 0
        o.cheb_guard = int(cheb_guard)
        self.precision = precision
        if isinstance(X0, torch.Tensor):
            x0p, x0dev = _dptr(X0, torch.float64, (A.n, p)), 1
        else:
            X0 = np.ascontiguousarray(X0, np.float64)
            self._keep.append(X0)
            x0p, x0dev = ctypes.c_void_p(X0.ctypes.data), 0
        self.n, self.p = int(A.n), int(p)
        self._stream = stream
        ctx = ctypes.c_void_p()
        _check(L.gsi_create(ctypes.byref(m), int(p), x0p, x0dev, ctypes.byref(o), _stream(stream),
                            ctypes.byref(ctx)), "gsi_create")
        self._ctx = ctx
        self._keep = []

    def step(self, nsteps=1):
        info = Info()
        _check(lib().gsi_step(self._ctx, int(nsteps), ctypes.byref(info)), "gsi_step")
        return info.as_dict()

    def set_operator(self, A, anorm=0.0):
        """gsi_set_operator: the next problem of a sequence (same n and format),
        started from the current iterate."""
        keep = []
        m = _matrix(A, self._fmt, keep)
        _check(lib().gsi_set_operator(self._ctx, ctypes.byref(m), float(anorm)), "gsi_set_operator")

    def solve(self, raise_on_noconv=False):
        info = Info()
        s = lib().gsi_solve(self._ctx, ctypes.byref(info))
        if s != GSI_OK and (s != GSI_ERR_NOCONV or raise_on_noconv):
            raise GsiError(s, "gsi_solve")
        return info.as_dict()

    def basis(self, evals=True, device=False):
        """(X, evals): Ritz vectors and values (evals=True), or the raw iterate."""
        import torch
        if device:
            X = torch.empty((self.n, self.p), dtype=torch.float64, device="cuda")
            ev = torch.empty(self.p, dtype=torch.float64, device="cuda") if evals else None
            _check(lib().gsi_get_basis(self._ctx, ctypes.c_void_p(X.data_ptr()),
                                       ctypes.c_void_p(ev.data_ptr()) if evals else None, 1),
                   "gsi_get_basis")
            return X, ev
        X = np.empty((self.n, self.p))
        ev = np.empty(self.p) if evals else None
        _check(lib().gsi_get_basis(self._ctx, ctypes.c_void_p(X.ctypes.data),
                                   ctypes.c_void_p(ev.ctypes.data) if evals else None, 0),
               "gsi_get_basis")
        return X, ev

    def state(self):
        """Zero-copy torch views of the current X and Y = AX (library memory):
        float64 (n, p) for precision 'f64', float32 (n, p, 2) df64 pairs otherwise."""
        import torch
        xp, yp = ctypes.c_void_p(), ctypes.c_void_p()
        _check(lib().gsi_state_ptrs(self._ctx, ctypes.byref(xp), ctypes.byref(yp)), "gsi_state_ptrs")
        if self.precision == "f64":
            shape, ts = (self.n, self.p), "<f8"
        else:
            shape, ts = (self.n, self.p, 2), "<f4"
        X = torch.as_tensor(_DeviceArray(xp.value, shape, ts), device="cuda")
        Y = torch.as_tensor(_DeviceArray(yp.value, shape, ts), device="cuda")
        return X, Y

    def reset(self, X0):
        import torch
        if isinstance(X0, torch.Tensor):
            _check(lib().gsi_reset(self._ctx, _dptr(X0, torch.float64, (self.n, self.p)), 1), "gsi_reset")
        else:
            X0 = np.ascontiguousarray(X0, np.float64)
            _check(lib().gsi_reset(self._ctx, ctypes.c_void_p(X0.ctypes.data), 0), "gsi_reset")

    def profile(self, on=True):
        _check(lib().gsi_profile_enable(self._ctx, 1 if on else 0), "gsi_profile_enable")

    def profile_read(self):
        """{class: {launches, ms, bytes, flops}} since profile(True)."""
        out = {}
        for k, name in enumerate(KERNEL_CLASSES):
            l, ms, b, f = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
            _check(lib().gsi_profile_read(self._ctx, k, ctypes.byref(l), ctypes.byref(ms),
                                          ctypes.byref(b), ctypes.byref(f)), "gsi_profile_read")
            out[name] = {"launches": l.value, "ms": ms.value, "bytes": b.value, "flops": f.value}
        return out

    def close(self):
        if getattr(self, "_ctx", None):
            lib().gsi_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def batched_plan(n, p, tile_max, target_tiles, active=None):
    """Host-only tile table of one pass of the batched solver:
    (order, [(problem, first row, rows), ...])."""
    L = lib()
    n = np.ascontiguousarray(n, np.int32)
    p = np.ascontiguousarray(p, np.int32)
    act = None if active is None else np.ascontiguousarray(active, np.int32)
    ap = None if act is None else act.ctypes.data
    nt = ctypes.c_int32()
    order = np.zeros(n.size, np.int32)
    _check(L.gsi_batched_plan(n.size, n.ctypes.data, p.ctypes.data, ap, int(tile_max), int(target_tiles),
                              order.ctypes.data, ctypes.byref(nt), None, None, None, 0), "gsi_batched_plan")
    cap = nt.value
    tp, t0, tr = (np.zeros(max(cap, 1), np.int32) for _ in range(3))
    _check(L.gsi_batched_plan(n.size, n.ctypes.data, p.ctypes.data, ap, int(tile_max), int(target_tiles),
                              None, ctypes.byref(nt), tp.ctypes.data, t0.ctypes.data, tr.ctypes.data, cap),
           "gsi_batched_plan")
    return order, list(zip(tp[:cap].tolist(), t0[:cap].tolist(), tr[:cap].tolist()))


class Batch:
    """gsi_batched_create / _tune / _step / _solve / _info / _get_basis.

    B: object with n, p (per problem), rowptr (global int64), colidx (local
    int32), val (float32) and X0 (concatenated float64 start blocks), as
    made by inputs.er_batch."""

    def __init__(self, B, method="cg", which=1, tol=1e-8, anorm=None, max_iters=10000,
                 k_restart=0, recompute_every=50, explicit_ax=False, stream=None):
        L = lib()
        self._keep = [np.ascontiguousarray(B.n, np.int32), np.ascontiguousarray(B.p, np.int32),
                      np.ascontiguousarray(B.rowptr, np.int64), np.ascontiguousarray(B.colidx, np.int32),
                      np.ascontiguousarray(B.val, np.float32), np.ascontiguousarray(B.X0, np.float64)]
        an = None
        if anorm is not None:
            an = np.ascontiguousarray(anorm, np.float64)
            self._keep.append(an)
        o = Opts()
        L.gsi_default_opts(ctypes.byref(o))
        o.method = {"sd": GSI_SD, "cg": GSI_CG}[method]
        o.which = int(which)
        o.tol = float(tol)
        o.max_iters = int(max_iters)
        o.k_restart = int(k_restart)
        o.recompute_every = int(recompute_every)
        o.explicit_ax = 1 if explicit_ax else 0
        self.n = self._keep[0].copy()
        self.p = self._keep[1].copy()
        self.nprob = int(self.n.size)
        self._stream = stream
        ctx = ctypes.c_void_p()
        _check(L.gsi_batched_create(self.nprob, *(a.ctypes.data for a in self._keep[:6]),
                                    None if an is None else an.ctypes.data, ctypes.byref(o),
                                    _stream(stream), ctypes.byref(ctx)), "gsi_batched_create")
        self._ctx = ctx

    def set_tiles(self, tile_max, ctas_per_sm, tiles_per_cta=2):
        _check(lib().gsi_batched_set_tiles(self._ctx, int(tile_max), int(ctas_per_sm), int(tiles_per_cta)),
               "gsi_batched_set_tiles")

    def tiles(self):
        a, b, c, d = (ctypes.c_int32() for _ in range(4))
        _check(lib().gsi_batched_get_tiles(self._ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                           ctypes.byref(d)), "gsi_batched_get_tiles")
        return {"tile_max": a.value, "ctas_per_sm": b.value, "tiles_per_cta": c.value, "grid": d.value}

    def last_plan(self):
        """The tile table the device built for the last pass."""
        nt = ctypes.c_int32()
        _check(lib().gsi_batched_last_plan(self._ctx, ctypes.byref(nt), None, None, None, 0),
               "gsi_batched_last_plan")
        cap = max(nt.value, 1)
        tp, t0, tr = (np.zeros(cap, np.int32) for _ in range(3))
        _check(lib().gsi_batched_last_plan(self._ctx, ctypes.byref(nt), tp.ctypes.data, t0.ctypes.data,
                                           tr.ctypes.data, cap), "gsi_batched_last_plan")
        k = nt.value
        return list(zip(tp[:k].tolist(), t0[:k].tolist(), tr[:k].tolist()))

    def tune(self, npasses=3):
        a, b, c, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
        _check(lib().gsi_batched_tune(self._ctx, int(npasses), ctypes.byref(a), ctypes.byref(b),
                                      ctypes.byref(c), ctypes.byref(ms)), "gsi_batched_tune")
        return {"tile_max": a.value, "ctas_per_sm": b.value, "tiles_per_cta": c.value,
                "ms_per_pass": ms.value}

    def reset(self):
        _check(lib().gsi_batched_reset(self._ctx), "gsi_batched_reset")

    def step(self, npasses=1):
        _check(lib().gsi_batched_step(self._ctx, int(npasses)), "gsi_batched_step")

    def solve(self, use_graph=True, check=True):
        """Run to the end; returns the number of passes. check=False keeps a
        GSI_ERR_NOCONV (some problem not converged) silent."""
        passes = ctypes.c_int32()
        st = lib().gsi_batched_solve(self._ctx, 1 if use_graph else 0, ctypes.byref(passes))
        if check or st != GSI_ERR_NOCONV:
            _check(st, "gsi_batched_solve")
        return passes.value

    def info(self, i):
        inf, st = Info(), ctypes.c_int32()
        _check(lib().gsi_batched_info(self._ctx, int(i), ctypes.byref(inf), ctypes.byref(st)),
               "gsi_batched_info")
        d = {k: getattr(inf, k) for k, _ in Info._fields_}
        d["status"] = st.value
        return d

    def basis(self, i, evals=True):
        X = np.zeros((int(self.n[i]), int(self.p[i])), np.float64)
        ev = np.zeros(int(self.p[i]), np.float64) if evals else None
        _check(lib().gsi_batched_get_basis(self._ctx, int(i), X.ctypes.data,
                                           None if ev is None else ev.ctypes.data),
               "gsi_batched_get_basis")
        return X, ev

    def restart(self, X0):
        """New start blocks (concatenated float64, numpy or torch CUDA)."""
        import torch
        if isinstance(X0, torch.Tensor):
            _check(lib().gsi_batched_restart(self._ctx, _dptr(X0, torch.float64), 1), "gsi_batched_restart")
        else:
            X0 = np.ascontiguousarray(X0, np.float64)
            _check(lib().gsi_batched_restart(self._ctx, X0.ctypes.data, 0), "gsi_batched_restart")

    def close(self):
        if getattr(self, "_ctx", None):
            lib().gsi_batched_destroy(self._ctx)
            self._ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- learned warm start --------------------------------------------------------

def mlp_num_params(din, hidden, dout):
    return int(lib().gsi_mlp_num_params(int(din), int(hidden), int(dout)))


def _f32(t):
    import torch
    return _dptr(t, torch.float32)


class MLP:
    """gsi_mlp_*: din -> hidden -> hidden -> dout, parameters as one float32
    vector W1, b1, W2, b2, W3, b3 (row-major)."""

    def __init__(self, din, hidden, dout, params, max_batch=256, stream=None):
        self.din, self.hidden, self.dout, self.max_batch = int(din), int(hidden), int(dout), int(max_batch)
        self.np = mlp_num_params(din, hidden, dout)
        flat = np.ascontiguousarray(params, np.float32).ravel()
        if flat.size != self.np:
            raise ValueError("params must hold %d floats" % self.np)
        ctx = ctypes.c_void_p()
        _check(lib().gsi_mlp_create(self.din, self.hidden, self.dout, self.max_batch, flat.ctypes.data,
                                    _stream(stream), ctypes.byref(ctx)), "gsi_mlp_create")
        self._ctx = ctx

    @staticmethod
    def flatten(prm):
        return np.concatenate([np.asarray(prm[k], np.float32).ravel()
                               for k in ("W1", "b1", "W2", "b2", "W3", "b3")])

    def unflatten(self, flat):
        d, h, o = self.din, self.hidden, self.dout
        out, k = {}, 0
        for name, shape in (("W1", (h, d)), ("b1", (h,)), ("W2", (h, h)), ("b2", (h,)),
                            ("W3", (o, h)), ("b3", (o,))):
            size = int(np.prod(shape))
            out[name] = flat[k:k + size].reshape(shape)
            k += size
        return out

    def params(self):
        w = np.zeros(self.np, np.float32)
        _check(lib().gsi_mlp_get_params(self._ctx, w.ctypes.data, None), "gsi_mlp_get_params")
        return self.unflatten(w)

    def grads(self):
        g = np.zeros(self.np, np.float32)
        _check(lib().gsi_mlp_get_params(self._ctx, None, g.ctypes.data), "gsi_mlp_get_params")
        return self.unflatten(g)

    def forward(self, x, out):
        _check(lib().gsi_mlp_forward(self._ctx, int(x.shape[0]), _f32(x), _f32(out)), "gsi_mlp_forward")
        return out

    def backward(self, x, dout):
        _check(lib().gsi_mlp_backward(self._ctx, int(x.shape[0]), _f32(x), _f32(dout)), "gsi_mlp_backward")

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        _check(lib().gsi_mlp_adam(self._ctx, float(lr), float(beta1), float(beta2), float(eps)),
               "gsi_mlp_adam")

    def train_step(self, x, S, Bt, m, p, lr):
        """forward, mean-loss gradient, backward, Adam; returns the mean loss.
        S = (rowptr int64, colidx int32, val float64) CUDA tensors."""
        import torch
        loss = ctypes.c_double()
        _check(lib().gsi_warm_train_step(self._ctx, int(x.shape[0]), _f32(x), int(m), int(p),
                                         _dptr(S[0], torch.int64), _dptr(S[1], torch.int32),
                                         _dptr(S[2], torch.float64), _f32(Bt), float(lr), ctypes.byref(loss)),
               "gsi_warm_train_step")
        return loss.value

    def close(self):
        if getattr(self, "_ctx", None):
            lib().gsi_mlp_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def warm_loss_grad(C, S, Bt, m, p, gscale=1.0, stream=None):
    """(loss (batch,), dC) for C, Bt (batch x m x p float32 CUDA tensors)."""
    import torch
    batch = int(C.shape[0])
    loss = torch.empty(batch, dtype=torch.float64, device=C.device)
    dC = torch.empty_like(C)
    SC = torch.empty_like(C)
    _check(lib().gsi_warm_loss_grad(batch, int(m), int(p), _dptr(S[0], torch.int64), _dptr(S[1], torch.int32),
                                    _dptr(S[2], torch.float64), _f32(C), _f32(Bt), _f32(SC),
                                    _dptr(loss, torch.float64), _f32(dC), ctypes.c_float(gscale),
                                    _stream(stream)), "gsi_warm_loss_grad")
    return loss, dC


def prolong(C, nc, nf, p, stream=None):
    """X (batch x nf^2 x p float64) = P C for C (batch x nc^2 x p float32)."""
    import torch
    batch = int(C.shape[0])
    X = torch.empty((batch, nf * nf, p), dtype=torch.float64, device=C.device)
    _check(lib().gsi_prolong(int(nc), int(nf), int(p), batch, _f32(C), _dptr(X, torch.float64),
                             _stream(stream)), "gsi_prolong")
    return X


def restrict(U, nc, nf, p, stream=None):
    """Bt (batch x nc^2 x p float32) = P^T U for U (batch x nf^2 x p float64)."""
    import torch
    batch = int(U.shape[0])
    Bt = torch.empty((batch, nc * nc, p), dtype=torch.float32, device=U.device)
    _check(lib().gsi_restrict(int(nc), int(nf), int(p), batch, _dptr(U, torch.float64), _f32(Bt),
                              _stream(stream)), "gsi_restrict")
    return Bt


def gemm_bf16(M, N, K, A, sa, B, sb, C, ldc, alpha=1.0, beta=0.0, bias=None, mask=None, relu=False,
              stream=None):
    """C = alpha op(A) op(B) + beta C (+ bias, mask, ReLU) with strides
    sa = (sai, sak), sb = (sbk, sbj); float32 CUDA tensors."""
    _check(lib().gsi_gemm_bf16(int(M), int(N), int(K), _f32(A), int(sa[0]), int(sa[1]), _f32(B), int(sb[0]),
                               int(sb[1]), _f32(C), int(ldc), ctypes.c_float(alpha), ctypes.c_float(beta),
                               None if bias is None else _f32(bias), None if mask is None else _f32(mask),
                               1 if relu else 0, _stream(stream)), "gsi_gemm_bf16")
    return C
