"""Python binding of the RHOSVD CUDA library (``include/rhosvd.h``).

Argument marshalling only: every step runs in the library's CUDA kernels.  PyTorch
provides device memory and the current stream.  The functions carry the C names:

    rhosvd_version, rhosvd_strerror, rhosvd_c2t_workspace_size, rhosvd_subspace_width,
    rhosvd_c2t, rhosvd_cp_hadamard, rhosvd_cp_sum

Factor matrices are column-major: a factor U^(l) is a float64 CUDA tensor of shape
(n_l, R) with stride (1, ld), e.g. ``torch.empty(R, n).t()``.  If the library cannot be
loaded (not built, no CUDA), every entry point raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
_lock = threading.Lock()
_lib = None

RHOSVD_OK = 0
RHOSVD_ERR_INVALID_ARG = -1
RHOSVD_ERR_RANK_OVERFLOW = -2
RHOSVD_ERR_NOT_CONVERGED = -3
RHOSVD_ERR_NONFINITE = -4
RHOSVD_ERR_SKETCH = -5
RHOSVD_ERR_CUDA = -6
RHOSVD_ERR_WORKSPACE = -7
RHOSVD_ERR_SCRATCH_LIMIT = -8
RHOSVD_NOALLOC_SCRATCH_BYTES = 64 << 20
RHOSVD_PLAIN_FP64 = 0
RHOSVD_MIXED = 1
RHOSVD_ERR_TIMEOUT = -9
RHOSVD_K_MAX = 256

_c = ctypes


class rhosvd_cp(_c.Structure):
    _fields_ = [("n", _c.c_int * 3), ("R", _c.c_int), ("U", _c.c_void_p * 3), ("ld", _c.c_int * 3),
                ("xi", _c.c_void_p)]


class rhosvd_opts(_c.Structure):
    _fields_ = [("eps", _c.c_double), ("ranks", _c.c_int * 3), ("r_max", _c.c_int), ("oversample", _c.c_int),
                ("precision", _c.c_int), ("deflate", _c.c_int), ("seed", _c.c_ulonglong), ("out_fp32", _c.c_int)]


class rhosvd_info(_c.Structure):
    _fields_ = [("status", _c.c_int), ("r", _c.c_int * 3), ("r_needed", _c.c_int * 3), ("k", _c.c_int * 3),
                ("kept", _c.c_int), ("direct", _c.c_int * 3), ("xi_norm", _c.c_double),
                ("total", _c.c_double * 3), ("resid", _c.c_double * 3), ("tail", _c.c_double * 3)]


class rhosvd_tucker(_c.Structure):
    _fields_ = [("Z", _c.c_void_p * 3), ("beta", _c.c_void_p), ("sigma", _c.c_void_p * 3), ("V", _c.c_void_p * 3),
                ("xi_out", _c.c_void_p), ("info", _c.c_void_p)]


class rhosvd_tucker_in(_c.Structure):
    _fields_ = [("n", _c.c_int * 3), ("r", _c.c_int * 3), ("Z", _c.c_void_p * 3), ("ldz", _c.c_int * 3),
                ("beta", _c.c_void_p)]


class rhosvd_horner_step(_c.Structure):
    _fields_ = [("k", _c.c_int), ("R_in", _c.c_int), ("r", _c.c_int * 3), ("R", _c.c_int), ("status", _c.c_int)]


class RhosvdError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        super().__init__(f"{where}: {rhosvd_strerror(code)} ({code})")


def lib_path() -> str:
    return os.path.join(_HERE, "_build", "librhosvd.so")


def load(build_if_missing: bool = False):
    """Load librhosvd.so (raises if it is missing or cannot be loaded)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"RHOSVD CUDA library not built ({path}); run __graft_entry__.build()")
            from . import build_lib
            build_lib.build()
        L = _c.CDLL(path)
        L.rhosvd_version.restype = _c.c_int
        L.rhosvd_strerror.restype = _c.c_char_p
        L.rhosvd_strerror.argtypes = [_c.c_int]
        L.rhosvd_c2t_workspace_size.restype = _c.c_size_t
        L.rhosvd_c2t_workspace_size.argtypes = [_c.POINTER(rhosvd_cp), _c.POINTER(rhosvd_opts)]
        L.rhosvd_subspace_width.restype = _c.c_int
        L.rhosvd_subspace_width.argtypes = [_c.POINTER(rhosvd_cp), _c.POINTER(rhosvd_opts), _c.c_int]
        L.rhosvd_c2t.restype = _c.c_int
        L.rhosvd_c2t.argtypes = [_c.POINTER(rhosvd_cp), _c.POINTER(rhosvd_opts), _c.POINTER(rhosvd_tucker),
                                 _c.c_void_p, _c.c_size_t, _c.c_void_p]
        L.rhosvd_cp_hadamard.restype = _c.c_int
        L.rhosvd_cp_hadamard.argtypes = [_c.POINTER(rhosvd_cp), _c.POINTER(rhosvd_cp), _c.c_void_p * 3,
                                         _c.c_int * 3, _c.c_void_p, _c.c_void_p]
        L.rhosvd_cp_sum.restype = _c.c_int
        L.rhosvd_cp_sum.argtypes = [_c.c_double, _c.POINTER(rhosvd_cp), _c.c_double, _c.POINTER(rhosvd_cp),
                                    _c.c_void_p * 3, _c.c_int * 3, _c.c_void_p, _c.c_void_p]
        L.rhosvd_c2t_noalloc.restype = _c.c_int
        L.rhosvd_c2t_noalloc.argtypes = [_c.POINTER(rhosvd_cp), _c.POINTER(rhosvd_opts), _c.POINTER(rhosvd_tucker),
                                         _c.c_void_p]
        L.rhosvd_c2t_batched_workspace_size.restype = _c.c_size_t
        L.rhosvd_c2t_batched_workspace_size.argtypes = [_c.c_int, _c.POINTER(rhosvd_cp), _c.POINTER(rhosvd_opts),
                                                        _c.c_int]
        L.rhosvd_c2t_batched.restype = _c.c_int
        L.rhosvd_c2t_batched.argtypes = [_c.c_int, _c.POINTER(rhosvd_cp), _c.POINTER(rhosvd_opts),
                                         _c.POINTER(rhosvd_tucker), _c.c_void_p, _c.c_size_t, _c.c_int, _c.c_void_p]
        L.rhosvd_batch_latency_enable.restype = _c.c_int
        L.rhosvd_batch_latency_enable.argtypes = [_c.c_int]
        L.rhosvd_batch_latency_read.restype = _c.c_int
        L.rhosvd_batch_latency_read.argtypes = [_c.POINTER(_c.c_float), _c.c_int]
        L.rhosvd_c2t_start_workspace_size.restype = _c.c_size_t
        L.rhosvd_c2t_start_workspace_size.argtypes = [_c.POINTER(rhosvd_cp), _c.POINTER(rhosvd_opts), _c.c_int]
        L.rhosvd_c2t_start.restype = _c.c_int
        L.rhosvd_c2t_start.argtypes = [_c.POINTER(rhosvd_cp), _c.POINTER(rhosvd_opts), _c.c_void_p * 3, _c.c_int * 3,
                                       _c.c_int, _c.c_int, _c.POINTER(rhosvd_tucker), _c.c_void_p, _c.c_size_t,
                                       _c.c_void_p]
        L.rhosvd_mlp_create.restype = _c.c_int
        L.rhosvd_mlp_create.argtypes = [_c.c_int, _c.c_ulonglong, _c.POINTER(_c.c_void_p)]
        L.rhosvd_mlp_destroy.restype = _c.c_int
        L.rhosvd_mlp_destroy.argtypes = [_c.c_void_p]
        L.rhosvd_mlp_forward.restype = _c.c_int
        L.rhosvd_mlp_forward.argtypes = [_c.c_void_p, _c.c_void_p, _c.c_int, _c.c_void_p, _c.c_void_p]
        L.rhosvd_mlp_gradients.restype = _c.c_int
        L.rhosvd_mlp_gradients.argtypes = [_c.c_void_p, _c.c_void_p, _c.c_void_p, _c.c_int, _c.c_void_p, _c.c_void_p]
        L.rhosvd_mlp_train_step.restype = _c.c_int
        L.rhosvd_mlp_train_step.argtypes = [_c.c_void_p, _c.c_void_p, _c.c_void_p, _c.c_int, _c.c_float, _c.c_void_p,
                                            _c.c_void_p]
        L.rhosvd_mlp_num_params.restype = _c.c_longlong
        L.rhosvd_mlp_params.restype = _c.c_int
        L.rhosvd_mlp_params.argtypes = [_c.c_void_p, _c.c_void_p, _c.c_int, _c.c_int]
        L.rhosvd_probe_fp64.restype = _c.c_int
        L.rhosvd_probe_fp64.argtypes = [_c.c_int, _c.c_int, _c.c_void_p, _c.c_void_p]
        L.rhosvd_mlp_save.restype = _c.c_int
        L.rhosvd_mlp_save.argtypes = [_c.c_void_p, _c.c_char_p]
        L.rhosvd_mlp_load.restype = _c.c_int
        L.rhosvd_mlp_load.argtypes = [_c.c_void_p, _c.c_char_p]
        L.rhosvd_mlp_status.restype = _c.c_int
        L.rhosvd_mlp_status.argtypes = [_c.c_void_p, _c.c_void_p]
        L.rhosvd_features.restype = _c.c_int
        L.rhosvd_features.argtypes = [_c.c_void_p, _c.c_void_p, _c.c_void_p, _c.c_int, _c.c_double, _c.c_double,
                                      _c.c_double, _c.c_void_p, _c.c_void_p]
        L.rhosvd_chebyshev.restype = _c.c_int
        L.rhosvd_chebyshev.argtypes = [_c.c_int, _c.c_double, _c.c_void_p, _c.c_void_p]
        L.rhosvd_proj_target.restype = _c.c_int
        L.rhosvd_proj_target.argtypes = [_c.c_int, _c.c_void_p, _c.c_void_p, _c.c_int, _c.c_int, _c.c_void_p,
                                         _c.c_void_p]
        L.rhosvd_proposal_basis.restype = _c.c_int
        L.rhosvd_proposal_basis.argtypes = [_c.c_int, _c.c_void_p, _c.c_void_p, _c.c_void_p, _c.c_void_p]
        L.rhosvd_t2c_workspace_size.restype = _c.c_size_t
        L.rhosvd_t2c_workspace_size.argtypes = [_c.POINTER(rhosvd_tucker_in)]
        L.rhosvd_t2c.restype = _c.c_int
        L.rhosvd_t2c.argtypes = [_c.POINTER(rhosvd_tucker_in), _c.c_double, _c.c_int, _c.c_void_p * 3, _c.c_int * 3,
                                 _c.c_void_p, _c.c_void_p, _c.c_void_p, _c.c_void_p, _c.c_void_p, _c.c_size_t,
                                 _c.c_void_p]
        L.rhosvd_c2t_als_workspace_size.restype = _c.c_size_t
        L.rhosvd_c2t_als_workspace_size.argtypes = [_c.POINTER(rhosvd_cp), _c.POINTER(rhosvd_opts), _c.c_int]
        L.rhosvd_c2t_als.restype = _c.c_int
        L.rhosvd_c2t_als.argtypes = [_c.POINTER(rhosvd_cp), _c.POINTER(rhosvd_opts), _c.c_int,
                                     _c.POINTER(rhosvd_tucker), _c.POINTER(_c.c_double), _c.c_void_p, _c.c_size_t,
                                     _c.c_void_p]
        L.rhosvd_c2t_hadamard_workspace_size.restype = _c.c_size_t
        L.rhosvd_c2t_hadamard_workspace_size.argtypes = [_c.POINTER(rhosvd_cp), _c.POINTER(rhosvd_cp),
                                                         _c.POINTER(rhosvd_opts)]
        L.rhosvd_c2t_hadamard.restype = _c.c_int
        L.rhosvd_c2t_hadamard.argtypes = [_c.POINTER(rhosvd_cp), _c.POINTER(rhosvd_cp), _c.POINTER(rhosvd_opts),
                                          _c.POINTER(rhosvd_tucker), _c.c_void_p, _c.c_size_t, _c.c_void_p]
        L.rhosvd_cp_sample.restype = _c.c_int
        L.rhosvd_cp_sample.argtypes = [_c.POINTER(rhosvd_cp), _c.c_int, _c.c_void_p, _c.c_void_p, _c.c_void_p]
        L.rhosvd_rs_energy.restype = _c.c_int
        L.rhosvd_rs_energy.argtypes = [_c.POINTER(rhosvd_cp), _c.c_int, _c.c_void_p, _c.c_void_p, _c.c_double,
                                       _c.c_void_p, _c.c_void_p, _c.c_void_p]
        L.rhosvd_cp_horner_workspace_size.restype = _c.c_size_t
        L.rhosvd_cp_horner_workspace_size.argtypes = [_c.POINTER(rhosvd_cp), _c.c_int, _c.POINTER(rhosvd_opts),
                                                      _c.c_int]
        L.rhosvd_cp_horner.restype = _c.c_int
        L.rhosvd_cp_horner.argtypes = [_c.POINTER(rhosvd_cp), _c.POINTER(_c.c_double), _c.c_int,
                                       _c.POINTER(rhosvd_opts), _c.c_double, _c.c_int, _c.c_void_p * 3,
                                       _c.c_int * 3, _c.c_void_p, _c.POINTER(_c.c_int),
                                       _c.POINTER(rhosvd_horner_step), _c.c_void_p, _c.c_size_t, _c.c_void_p]
        L.rhosvd_selftest_fastmath.restype = _c.c_int
        L.rhosvd_selftest_fastmath.argtypes = [_c.c_void_p, _c.c_void_p, _c.c_void_p, _c.c_int, _c.c_void_p]
        L.rhosvd_selftest_bits.restype = _c.c_int
        L.rhosvd_selftest_bits.argtypes = [_c.c_void_p] * 7 + [_c.c_int, _c.c_void_p]
        L.rhosvd_launch_count.restype = _c.c_longlong
        L.rhosvd_profile_enable.restype = _c.c_int
        L.rhosvd_profile_enable.argtypes = [_c.c_int]
        L.rhosvd_graph_begin.restype = _c.c_int
        L.rhosvd_graph_begin.argtypes = [_c.c_void_p]
        L.rhosvd_graph_end.restype = _c.c_int
        L.rhosvd_graph_end.argtypes = [_c.c_void_p, _c.POINTER(_c.c_void_p)]
        L.rhosvd_graph_launch.restype = _c.c_int
        L.rhosvd_graph_launch.argtypes = [_c.c_void_p, _c.c_void_p]
        L.rhosvd_graph_destroy.restype = _c.c_int
        L.rhosvd_graph_destroy.argtypes = [_c.c_void_p]
        L.rhosvd_profile_keep.restype = _c.c_int
        L.rhosvd_profile_keep.argtypes = [_c.c_int]
        L.rhosvd_profile_filter.restype = _c.c_int
        L.rhosvd_profile_filter.argtypes = [_c.c_char_p]
        L.rhosvd_profile_read.restype = _c.c_int
        L.rhosvd_profile_read.argtypes = [_c.c_char_p, _c.c_int]
        _lib = L
        return L


# ------------------------------------------------------------------ marshalling helpers

def _torch():
    import torch
    return torch


def _check_factor(U, l):
    torch = _torch()
    if not isinstance(U, torch.Tensor) or U.dtype != torch.float64 or U.dim() != 2 or not U.is_cuda:
        raise TypeError(f"factor {l} must be a 2-D float64 CUDA tensor")
    n, R = U.shape
    if R > 1 and n > 0 and U.stride(0) != 1:
        raise ValueError(f"factor {l} must be column-major (stride (1, ld)); got stride {tuple(U.stride())}")
    ld = U.stride(1) if R > 1 else max(n, 1)
    return n, R, max(ld, n)


def make_cp(U, xi) -> rhosvd_cp:
    cp = rhosvd_cp()
    R = None
    for l in range(3):
        n, Rl, ld = _check_factor(U[l], l)
        if R is None:
            R = Rl
        elif Rl != R:
            raise ValueError("factors disagree on the rank R")
        cp.n[l] = n
        cp.ld[l] = ld
        cp.U[l] = U[l].data_ptr()
    if xi.dtype != _torch().float64 or not xi.is_cuda or xi.numel() != R or not xi.is_contiguous():
        raise ValueError("xi must be a contiguous float64 CUDA tensor of length R")
    cp.R = R
    cp.xi = xi.data_ptr()
    return cp


def make_opts(eps=1e-6, ranks=(0, 0, 0), r_max=64, oversample=32, seed=0,
              precision=RHOSVD_PLAIN_FP64, deflate=0, out_fp32=False) -> rhosvd_opts:
    o = rhosvd_opts()
    o.out_fp32 = 1 if out_fp32 else 0
    o.eps = float(eps)
    for l in range(3):
        o.ranks[l] = int(ranks[l])
    o.r_max = int(r_max)
    o.oversample = int(oversample)
    o.precision = int(precision)
    o.deflate = int(deflate)
    o.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return o


def _stream_handle(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return _c.c_void_p(s.cuda_stream)


# ------------------------------------------------------------------ C entry points

def rhosvd_version() -> int:
    return int(load().rhosvd_version())


def rhosvd_strerror(code: int) -> str:
    try:
        return load().rhosvd_strerror(int(code)).decode()
    except Exception:                                  # library unavailable
        return f"status {code}"


@dataclass
class CanonicalResult:
    """Device outputs of one rhosvd_t2c call: factors U[l] (n_l x R_max, column-major), weights
    xi, and device ints R (canonical rank), status, p (per slice)."""
    U: list
    xi: object
    R_dev: object
    status_dev: object
    p: object

    def rank(self):
        """Synchronise the current stream; (R, status)."""
        torch = _torch()
        torch.cuda.current_stream().synchronize()
        return int(self.R_dev.item()), int(self.status_dev.item())


def rhosvd_t2c(Z, beta, eps, R_max, workspace=None, stream=None, out=None) -> CanonicalResult:
    """Tucker-to-canonical transform.  Z: three column-major float64 CUDA matrices (n_l x r_l);
    beta: float64 CUDA tensor of r1*r2*r3 entries, (i, j, m) at i + r1 (j + r2 m)."""
    torch = _torch()
    L = load()
    t = rhosvd_tucker_in()
    r = [int(z.shape[1]) for z in Z]
    for l in range(3):
        t.n[l] = int(Z[l].shape[0])
        t.r[l] = r[l]
        t.Z[l] = Z[l].data_ptr()
        t.ldz[l] = int(Z[l].stride(1)) if r[l] > 1 else max(int(Z[l].shape[0]), 1)
        if r[l] > 0 and Z[l].stride(0) != 1:
            raise ValueError("Z must be column-major")
    t.beta = beta.data_ptr() if beta.numel() else None
    need = int(L.rhosvd_t2c_workspace_size(_c.byref(t)))
    if need == 0:
        raise RhosvdError(RHOSVD_ERR_INVALID_ARG, "rhosvd_t2c_workspace_size")
    dev = Z[0].device
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=dev)
    cap = max(int(R_max), 0)
    if out is not None:           # reuse the buffers of an earlier call (same shapes, capacity >= R_max)
        U, xi, R_dev, st_dev, p = out.U, out.xi, out.R_dev, out.status_dev, out.p
    else:
        U = [torch.empty(max(cap, 1), t.n[l], dtype=torch.float64, device=dev).t() for l in range(3)]
        xi = torch.empty(max(cap, 1), dtype=torch.float64, device=dev)
        R_dev = torch.zeros(1, dtype=torch.int32, device=dev)
        st_dev = torch.zeros(1, dtype=torch.int32, device=dev)
        p = torch.zeros(max(r[2], 1), dtype=torch.int32, device=dev)
    ptrs = (_c.c_void_p * 3)(*[U[l].data_ptr() for l in range(3)])
    ldu = (_c.c_int * 3)(*[max(t.n[l], 1) for l in range(3)])
    rc = L.rhosvd_t2c(_c.byref(t), float(eps), cap, ptrs, ldu, _c.c_void_p(xi.data_ptr()),
                      _c.c_void_p(R_dev.data_ptr()), _c.c_void_p(p.data_ptr()), _c.c_void_p(st_dev.data_ptr()),
                      _c.c_void_p(workspace.data_ptr()), need, _stream_handle(stream))
    if rc != RHOSVD_OK:
        raise RhosvdError(rc, "rhosvd_t2c")
    return CanonicalResult(U=U, xi=xi, R_dev=R_dev, status_dev=st_dev, p=p)


def rhosvd_c2c(U, xi, eps_tucker, eps_t2c, R_max, **c2t_opts):
    """Canonical-to-canonical reduction: rhosvd_c2t, then rhosvd_t2c of its Tucker tensor.
    Returns (CanonicalResult, TuckerResult)."""
    tk = rhosvd_c2t(U, xi, eps=eps_tucker, **c2t_opts)
    r, beta, Z = tk.tucker()
    flat = tk.beta[: r[0] * r[1] * r[2]]
    return rhosvd_t2c(Z, flat, eps_t2c, R_max), tk


class PolynomialResult:
    """Outputs of rhosvd_cp_horner: factors U[l] (n_l x R_max, column-major; columns < R hold
    P(A)), weights xi, the rank R and one record per reduction (dicts k, R_in, r, R, status)."""

    def __init__(self, U, xi, R, steps):
        self.U, self.xi, self.R, self.steps = U, xi, R, steps


def rhosvd_cp_horner(U, xi, coeffs, eps_tucker, eps_t2c, R_max, r_max=64, oversample=32, seed=0,
                     precision=RHOSVD_PLAIN_FP64, deflate=0, workspace=None, stream=None, out=None):
    """P(A) = sum_k coeffs[k] A^k (Hadamard powers) of the CP tensor A = (U, xi) by the Horner
    scheme with a C2C reduction after every product.  Synchronises the stream.  Raises
    RhosvdError on a host or device error (the records up to it are in err.steps)."""
    torch = _torch()
    L = load()
    cp = make_cp(U, xi)
    opts = make_opts(eps_tucker, (0, 0, 0), r_max, oversample, seed, precision, deflate)
    c = [float(a) for a in coeffs]
    nc = len(c)
    need = int(L.rhosvd_cp_horner_workspace_size(_c.byref(cp), nc, _c.byref(opts), int(R_max)))
    if need == 0:
        raise RhosvdError(RHOSVD_ERR_INVALID_ARG, "rhosvd_cp_horner_workspace_size")
    dev = U[0].device
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=dev)
    if out is None:
        Uo = [torch.empty(int(R_max), cp.n[l], dtype=torch.float64, device=dev).t() for l in range(3)]
        xo = torch.empty(int(R_max), dtype=torch.float64, device=dev)
    else:
        Uo, xo = out
    ptrs = (_c.c_void_p * 3)(*[Uo[l].data_ptr() for l in range(3)])
    ldu = (_c.c_int * 3)(*[cp.n[l] for l in range(3)])
    for l in range(3):
        if Uo[l].stride(0) != 1 or (Uo[l].shape[1] > 1 and Uo[l].stride(1) != cp.n[l]):
            raise ValueError("output factors must be column-major with leading dimension n_l")
    carr = (_c.c_double * nc)(*c)
    steps = (rhosvd_horner_step * max(nc - 1, 1))()
    for s in steps:
        s.k = -1                                  # records the call fills have k >= 0
    R = _c.c_int(0)
    rc = L.rhosvd_cp_horner(_c.byref(cp), carr, nc, _c.byref(opts), float(eps_t2c), int(R_max), ptrs, ldu,
                            _c.c_void_p(xo.data_ptr()), _c.byref(R), steps, _c.c_void_p(workspace.data_ptr()), need,
                            _stream_handle(stream))
    recs = [dict(k=s.k, R_in=s.R_in, r=list(s.r), R=s.R, status=s.status) for s in steps[: max(nc - 1, 0)]
            if s.k >= 0]
    if rc != RHOSVD_OK:
        err = RhosvdError(rc, "rhosvd_cp_horner")
        err.steps = recs
        raise err
    return PolynomialResult(Uo, xo, int(R.value), recs)


def _node_index(idx):
    """(N, 3) integer grid indices -> device int32 array of 3 N, mode-major."""
    torch = _torch()
    t = idx if isinstance(idx, torch.Tensor) else torch.as_tensor(idx)
    return t.to(device="cuda", dtype=torch.int32).t().contiguous().reshape(-1)


def rhosvd_cp_sample(U, xi, idx, out=None, stream=None):
    """Entries of the CP tensor (U, xi) at the (N, 3) grid indices idx; float64 CUDA tensor of N."""
    torch = _torch()
    L = load()
    cp = make_cp(U, xi)
    ix = _node_index(idx)
    N = ix.numel() // 3
    if out is None:
        out = torch.empty(max(N, 1), dtype=torch.float64, device=U[0].device)
    rc = L.rhosvd_cp_sample(_c.byref(cp), N, _c.c_void_p(ix.data_ptr()), _c.c_void_p(out.data_ptr()),
                            _stream_handle(stream))
    if rc != RHOSVD_OK:
        raise RhosvdError(rc, "rhosvd_cp_sample")
    return out[:N]


def rhosvd_rs_energy(U, xi, idx, z, p0, stream=None):
    """Interaction energy of the charges z (CUDA float64, N) at the grid nodes idx from the
    long-range potential (U, xi); returns (energy device scalar tensor, samples)."""
    torch = _torch()
    L = load()
    cp = make_cp(U, xi)
    ix = _node_index(idx)
    N = ix.numel() // 3
    p = torch.empty(max(N, 1), dtype=torch.float64, device=U[0].device)
    E = torch.empty(1, dtype=torch.float64, device=U[0].device)
    rc = L.rhosvd_rs_energy(_c.byref(cp), N, _c.c_void_p(ix.data_ptr()), _c.c_void_p(z.data_ptr()), float(p0),
                            _c.c_void_p(p.data_ptr()), _c.c_void_p(E.data_ptr()), _stream_handle(stream))
    if rc != RHOSVD_OK:
        raise RhosvdError(rc, "rhosvd_rs_energy")
    return E, p[:N]


def rhosvd_selftest_fastmath(x, stream=None):
    """(1/x, 1/sqrt(x)) by the library's short-latency device helpers (float64 CUDA tensor x)."""
    torch = _torch()
    x = x.contiguous()
    rcp, rsq = torch.empty_like(x), torch.empty_like(x)
    rc = load().rhosvd_selftest_fastmath(_c.c_void_p(x.data_ptr()), _c.c_void_p(rcp.data_ptr()),
                                         _c.c_void_p(rsq.data_ptr()), int(x.numel()), _stream_handle(stream))
    if rc != RHOSVD_OK:
        raise RhosvdError(rc, "rhosvd_selftest_fastmath")
    return rcp, rsq


def rhosvd_selftest_bits(x, f, e, stream=None):
    """(rh, rl, fd, p2) by the library's bit-level conversions: x float64, f float32, e int32 CUDA
    tensors of one length; rh + rl ~ x, fd = f 2^e (float64), p2 = 2^e (float32)."""
    torch = _torch()
    x, f, e = x.contiguous(), f.contiguous(), e.contiguous()
    n = int(x.numel())
    if f.numel() != n or e.numel() != n:
        raise RhosvdError(RHOSVD_ERR_INVALID_ARG, "rhosvd_selftest_bits: lengths differ")
    rh = torch.empty(n, dtype=torch.float32, device=x.device)
    rl, p2 = torch.empty_like(rh), torch.empty_like(rh)
    fd = torch.empty(n, dtype=torch.float64, device=x.device)
    ptr = lambda t: _c.c_void_p(t.data_ptr())
    rc = load().rhosvd_selftest_bits(ptr(x), ptr(f), ptr(e), ptr(rh), ptr(rl), ptr(fd), ptr(p2), n,
                                     _stream_handle(stream))
    if rc != RHOSVD_OK:
        raise RhosvdError(rc, "rhosvd_selftest_bits")
    return rh, rl, fd, p2


def rhosvd_launch_count() -> int:
    return int(load().rhosvd_launch_count())


def rhosvd_profile_enable(on: bool) -> bool:
    return bool(load().rhosvd_profile_enable(1 if on else 0))


class Graph:
    """A captured sequence of library calls (see rhosvd_graph_begin); replay() launches it."""

    def __init__(self, handle):
        self.handle = handle

    def replay(self, stream=None):
        rc = load().rhosvd_graph_launch(self.handle, _stream_handle(stream))
        if rc != RHOSVD_OK:
            raise RhosvdError(rc, "rhosvd_graph_launch")

    def close(self):
        if self.handle:
            load().rhosvd_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rhosvd_capture(fn, stream):
    """Run fn() under capture on `stream` (a torch.cuda.Stream, not the default stream); returns
    a Graph replaying the library kernels fn launched."""
    L = load()
    h = _stream_handle(stream)
    rc = L.rhosvd_graph_begin(h)
    if rc != RHOSVD_OK:
        raise RhosvdError(rc, "rhosvd_graph_begin")
    try:
        fn()
    finally:
        g = _c.c_void_p()
        rc = L.rhosvd_graph_end(h, _c.byref(g))
    if rc != RHOSVD_OK:
        raise RhosvdError(rc, "rhosvd_graph_end")
    return Graph(g.value)


def rhosvd_profile_keep(on=True) -> int:
    """Keep the recorded stage events across reads (graph replays re-record them)."""
    return int(load().rhosvd_profile_keep(1 if on else 0))


def rhosvd_profile_filter(stage=None) -> int:
    """Time only the stages named `stage` (None: every stage)."""
    return int(load().rhosvd_profile_filter(stage.encode() if stage else None))


def rhosvd_profile_read() -> dict:
    """{stage: (count, total_ms)} accumulated since the last read (synchronises events)."""
    buf = _c.create_string_buffer(1 << 16)
    n = load().rhosvd_profile_read(buf, len(buf))
    if n < 0:
        raise RhosvdError(n, "rhosvd_profile_read")
    out = {}
    for line in buf.value.decode().splitlines():
        name, cnt, ms = line.split()
        out[name] = (int(cnt), float(ms))
    return out


def rhosvd_c2t_workspace_size(cp: rhosvd_cp, opts: rhosvd_opts) -> int:
    return int(load().rhosvd_c2t_workspace_size(_c.byref(cp), _c.byref(opts)))


def rhosvd_subspace_width(cp: rhosvd_cp, opts: rhosvd_opts, mode: int) -> int:
    return int(load().rhosvd_subspace_width(_c.byref(cp), _c.byref(opts), int(mode)))


@dataclass
class TuckerResult:
    """Device outputs of one rhosvd_c2t call (see rhosvd_tucker in include/rhosvd.h)."""
    Z: list
    beta: object
    sigma: object
    V: list
    xi_out: object
    info_buf: object
    r_max: int

    def info(self) -> rhosvd_info:
        """Synchronise the current stream and read the device-written info record."""
        torch = _torch()
        torch.cuda.current_stream().synchronize()
        raw = bytes(self.info_buf.cpu().numpy().tobytes())
        return rhosvd_info.from_buffer_copy(raw)

    def tucker(self):
        """(ranks, beta (r1,r2,r3) float64 CUDA view, [Z_l (n_l, r_l)])."""
        inf = self.info()
        r = [inf.r[l] for l in range(3)]
        cnt = r[0] * r[1] * r[2]
        beta = self.beta[:cnt].reshape(r[2], r[1], r[0]).permute(2, 1, 0)
        Z = [self.Z[l][:, : r[l]] for l in range(3)]
        return r, beta, Z


def alloc_tucker(n, R, r_max, device="cuda", with_V=False, with_xi=False, fp32=False) -> TuckerResult:
    """Output buffers of one reduction; fp32=True gives float32 Z and beta (opts.out_fp32)."""
    torch = _torch()
    zt = torch.float32 if fp32 else torch.float64
    Z = [torch.empty(r_max, n[l], dtype=zt, device=device).t() for l in range(3)]
    beta = torch.empty(r_max ** 3, dtype=zt, device=device)
    sigma = torch.empty(3, RHOSVD_K_MAX, dtype=torch.float64, device=device)
    V = [torch.empty(max(R, 1), r_max, dtype=torch.float64, device=device).t() for _ in range(3)] if with_V else None
    xi_out = torch.empty(max(R, 1), dtype=torch.float64, device=device) if with_xi else None
    info = torch.zeros(_c.sizeof(rhosvd_info), dtype=torch.uint8, device=device)
    return TuckerResult(Z=Z, beta=beta, sigma=sigma, V=V, xi_out=xi_out, info_buf=info, r_max=r_max)


def tucker_struct(res: TuckerResult) -> rhosvd_tucker:
    t = rhosvd_tucker()
    for l in range(3):
        t.Z[l] = res.Z[l].data_ptr()
        t.sigma[l] = res.sigma[l].data_ptr()
        t.V[l] = res.V[l].data_ptr() if res.V is not None else None
    t.beta = res.beta.data_ptr()
    t.xi_out = res.xi_out.data_ptr() if res.xi_out is not None else None
    t.info = res.info_buf.data_ptr()
    return t


def _check_out_dtype(out, out_fp32):
    torch = _torch()
    want = torch.float32 if out_fp32 else torch.float64
    if out.beta.dtype != want or any(z.dtype != want for z in out.Z):
        raise ValueError(f"Z and beta buffers must be {want} (out_fp32={bool(out_fp32)})")


def rhosvd_c2t(U, xi, eps=1e-6, ranks=(0, 0, 0), r_max=64, oversample=32, seed=0, out=None,
               workspace=None, stream=None, with_V=False, with_xi=False,
               precision=RHOSVD_PLAIN_FP64, deflate=0, out_fp32=False) -> TuckerResult:
    """RHOSVD canonical-to-Tucker transform of the CP tensor (U[0], U[1], U[2], xi).
    out_fp32=True writes Z and beta as float32 (sigma, V, xi' stay float64)."""
    torch = _torch()
    L = load()
    cp = make_cp(U, xi)
    opts = make_opts(eps, ranks, r_max, oversample, seed, precision, deflate, out_fp32)
    need = int(L.rhosvd_c2t_workspace_size(_c.byref(cp), _c.byref(opts)))
    if need == 0:
        raise RhosvdError(RHOSVD_ERR_INVALID_ARG, "rhosvd_c2t_workspace_size")
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=U[0].device)
    if out is None:
        out = alloc_tucker([cp.n[l] for l in range(3)], cp.R, r_max, U[0].device, with_V, with_xi, out_fp32)
    _check_out_dtype(out, out_fp32)
    t = tucker_struct(out)
    rc = L.rhosvd_c2t(_c.byref(cp), _c.byref(opts), _c.byref(t), _c.c_void_p(workspace.data_ptr()),
                      _c.c_size_t(workspace.numel()), _stream_handle(stream))
    if rc != RHOSVD_OK:
        raise RhosvdError(rc, "rhosvd_c2t")
    return out


def rhosvd_c2t_als(U, xi, sweeps=1, eps=1e-6, ranks=(0, 0, 0), r_max=64, oversample=32, seed=0, out=None,
                   workspace=None, stream=None, with_V=False, with_xi=False, precision=RHOSVD_PLAIN_FP64,
                   deflate=0, energies=True):
    """RHOSVD followed by `sweeps` ALS sweeps.  Returns (TuckerResult, energies) where energies is
    a list of (before, after) captured energies ||beta||^2 per mode step (the call then
    synchronises), or None with energies=False."""
    torch = _torch()
    L = load()
    cp = make_cp(U, xi)
    opts = make_opts(eps, ranks, r_max, oversample, seed, precision, deflate)
    need = int(L.rhosvd_c2t_als_workspace_size(_c.byref(cp), _c.byref(opts), int(sweeps)))
    if need == 0:
        raise RhosvdError(RHOSVD_ERR_INVALID_ARG, "rhosvd_c2t_als_workspace_size")
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=U[0].device)
    if out is None:
        out = alloc_tucker([cp.n[l] for l in range(3)], cp.R, r_max, U[0].device, with_V, with_xi)
    t = tucker_struct(out)
    e = (_c.c_double * max(6 * int(sweeps), 1))() if energies else None
    rc = L.rhosvd_c2t_als(_c.byref(cp), _c.byref(opts), int(sweeps), _c.byref(t), e,
                          _c.c_void_p(workspace.data_ptr()), _c.c_size_t(workspace.numel()), _stream_handle(stream))
    if rc != RHOSVD_OK:
        raise RhosvdError(rc, "rhosvd_c2t_als")
    hist = [(e[2 * s], e[2 * s + 1]) for s in range(3 * int(sweeps))] if energies else None
    return out, hist


def rhosvd_c2t_hadamard(Ua, xa, Ub, xb, eps=1e-6, ranks=(0, 0, 0), r_max=64, oversample=32, seed=0, out=None,
                        workspace=None, stream=None, with_V=False, with_xi=False, precision=RHOSVD_PLAIN_FP64,
                        deflate=0, out_fp32=False) -> TuckerResult:
    """RHOSVD of the Hadamard product of the CP tensors (Ua, xa) and (Ub, xb), the product's
    columns formed as they are read (bit-identical to rhosvd_cp_hadamard + rhosvd_c2t)."""
    torch = _torch()
    L = load()
    a, b = make_cp(Ua, xa), make_cp(Ub, xb)
    opts = make_opts(eps, ranks, r_max, oversample, seed, precision, deflate, out_fp32)
    need = int(L.rhosvd_c2t_hadamard_workspace_size(_c.byref(a), _c.byref(b), _c.byref(opts)))
    if need == 0:
        raise RhosvdError(RHOSVD_ERR_INVALID_ARG, "rhosvd_c2t_hadamard_workspace_size")
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=Ua[0].device)
    if out is None:
        out = alloc_tucker([a.n[l] for l in range(3)], a.R * b.R, r_max, Ua[0].device, with_V, with_xi, out_fp32)
    _check_out_dtype(out, out_fp32)
    t = tucker_struct(out)
    rc = L.rhosvd_c2t_hadamard(_c.byref(a), _c.byref(b), _c.byref(opts), _c.byref(t),
                               _c.c_void_p(workspace.data_ptr()), _c.c_size_t(workspace.numel()),
                               _stream_handle(stream))
    if rc != RHOSVD_OK:
        raise RhosvdError(rc, "rhosvd_c2t_hadamard")
    return out


def rhosvd_c2t_noalloc(U, xi, out, eps=1e-6, ranks=(0, 0, 0), r_max=64, oversample=32, seed=0,
                       stream=None, precision=RHOSVD_PLAIN_FP64, deflate=0, out_fp32=False) -> TuckerResult:
    """rhosvd_c2t without a workspace argument, for callers that cannot allocate device memory:
    the library uses its own static scratch array (RHOSVD_NOALLOC_SCRATCH_BYTES).  `out` must
    be provided (see alloc_tucker); this function allocates nothing."""
    L = load()
    cp = make_cp(U, xi)
    opts = make_opts(eps, ranks, r_max, oversample, seed, precision, deflate, out_fp32)
    _check_out_dtype(out, out_fp32)
    t = tucker_struct(out)
    rc = L.rhosvd_c2t_noalloc(_c.byref(cp), _c.byref(opts), _c.byref(t), _stream_handle(stream))
    if rc != RHOSVD_OK:
        raise RhosvdError(rc, "rhosvd_c2t_noalloc")
    return out


def _out_arrays(U_out):
    ptrs = (_c.c_void_p * 3)(*[u.data_ptr() for u in U_out])
    lds = (_c.c_int * 3)(*[max(u.stride(1) if u.shape[1] > 1 else u.shape[0], u.shape[0]) for u in U_out])
    return ptrs, lds


def rhosvd_cp_hadamard(Ua, xa, Ub, xb, U_out=None, xi_out=None, stream=None):
    """Hadamard product of two CP tensors; returns (U_out list, xi_out)."""
    torch = _torch()
    L = load()
    a, b = make_cp(Ua, xa), make_cp(Ub, xb)
    R = a.R * b.R
    dev = Ua[0].device
    if U_out is None:
        U_out = [torch.empty(R, a.n[l], dtype=torch.float64, device=dev).t() for l in range(3)]
    if xi_out is None:
        xi_out = torch.empty(R, dtype=torch.float64, device=dev)
    ptrs, lds = _out_arrays(U_out)
    rc = L.rhosvd_cp_hadamard(_c.byref(a), _c.byref(b), ptrs, lds, _c.c_void_p(xi_out.data_ptr()),
                              _stream_handle(stream))
    if rc != RHOSVD_OK:
        raise RhosvdError(rc, "rhosvd_cp_hadamard")
    return U_out, xi_out


def rhosvd_cp_sum(alpha, Ua, xa, beta, Ub, xb, U_out=None, xi_out=None, stream=None):
    """alpha A + beta B as one CP tensor; returns (U_out list, xi_out)."""
    torch = _torch()
    L = load()
    a, b = make_cp(Ua, xa), make_cp(Ub, xb)
    R = a.R + b.R
    dev = Ua[0].device
    if U_out is None:
        U_out = [torch.empty(R, a.n[l], dtype=torch.float64, device=dev).t() for l in range(3)]
    if xi_out is None:
        xi_out = torch.empty(R, dtype=torch.float64, device=dev)
    ptrs, lds = _out_arrays(U_out)
    rc = L.rhosvd_cp_sum(_c.c_double(alpha), _c.byref(a), _c.c_double(beta), _c.byref(b), ptrs, lds,
                         _c.c_void_p(xi_out.data_ptr()), _stream_handle(stream))
    if rc != RHOSVD_OK:
        raise RhosvdError(rc, "rhosvd_cp_sum")
    return U_out, xi_out


def to_device_factor(U_np, device="cuda"):
    """Column-major float64 CUDA copy of a numpy (n, R) array."""
    torch = _torch()
    import numpy as np
    a = np.asarray(U_np, dtype=np.float64)
    return torch.from_numpy(np.ascontiguousarray(a.T)).to(device).t()


class BatchedCall:
    """Marshalled arguments of one rhosvd_c2t_batched call (arrays of rhosvd_cp, rhosvd_opts and
    rhosvd_tucker plus the workspace).  Keep it and call run() again to repeat the same batch:
    the library then replays its cached graph."""

    def __init__(self, tensors, outs, lanes=0, device="cuda", **opt_kw):
        torch = _torch()
        L = load()
        self.count = len(tensors)
        self.cps = (rhosvd_cp * self.count)(*[make_cp(U, xi) for U, xi in tensors])
        self.opts = (rhosvd_opts * self.count)(*[make_opts(**opt_kw) for _ in range(self.count)])
        self.outs = outs
        self.tk = (rhosvd_tucker * self.count)(*[tucker_struct(o) for o in outs])
        self.lanes = int(lanes)
        need = int(L.rhosvd_c2t_batched_workspace_size(self.count, self.cps, self.opts, self.lanes))
        if need == 0:
            raise RhosvdError(RHOSVD_ERR_INVALID_ARG, "rhosvd_c2t_batched_workspace_size")
        self.workspace = torch.empty(need, dtype=torch.uint8, device=device)
        self._keep = tensors          # the factors must outlive the cached graph's use of them

    def run(self, stream=None):
        L = load()
        rc = L.rhosvd_c2t_batched(self.count, self.cps, self.opts, self.tk, _c.c_void_p(self.workspace.data_ptr()),
                                  _c.c_size_t(self.workspace.numel()), self.lanes, _stream_handle(stream))
        if rc != RHOSVD_OK:
            raise RhosvdError(rc, "rhosvd_c2t_batched")
        return self.outs


def rhosvd_c2t_batched(tensors, r_max=64, lanes=0, stream=None, with_V=False, with_xi=False, **opt_kw):
    """Reduce a list of canonical tensors [(U, xi), ...] in one batched call; returns the list of
    TuckerResult (one per tensor, as rhosvd_c2t would give) and the BatchedCall for repeats."""
    outs = [alloc_tucker([U[l].shape[0] for l in range(3)], U[0].shape[1], r_max, U[0].device, with_V, with_xi)
            for U, _ in tensors]
    call = BatchedCall(tensors, outs, lanes=lanes, device=tensors[0][0][0].device, r_max=r_max, **opt_kw)
    call.run(stream)
    return outs, call


def rhosvd_batch_latency_enable(on=True) -> int:
    return int(load().rhosvd_batch_latency_enable(1 if on else 0))


def rhosvd_batch_latency_read(count):
    """Completion time (ms since the batch started) of each tensor of the last batched call."""
    buf = (_c.c_float * count)()
    rc = load().rhosvd_batch_latency_read(buf, count)
    if rc != RHOSVD_OK:
        raise RhosvdError(rc, "rhosvd_batch_latency_read")
    return [float(x) for x in buf]


# ------------------------------------------------------------------ learned subspace proposal

def rhosvd_c2t_start(U, xi, Q0, iters=1, eps=1e-6, ranks=(0, 0, 0), r_max=64, oversample=32, seed=0, out=None,
                     workspace=None, stream=None, with_V=False, with_xi=False, precision=RHOSVD_PLAIN_FP64,
                     deflate=0) -> TuckerResult:
    """rhosvd_c2t with the range sketch replaced by the start basis Q0 (list of three n_l x k0
    column-major float64 CUDA tensors): iters 0 uses Q0 itself, iters 1 one subspace iteration."""
    torch = _torch()
    L = load()
    cp = make_cp(U, xi)
    opts = make_opts(eps, ranks, r_max, oversample, seed, precision, deflate)
    k0 = int(Q0[0].shape[1])
    q = (_c.c_void_p * 3)()
    ld = (_c.c_int * 3)()
    for l in range(3):
        if Q0[l].dtype != torch.float64 or Q0[l].shape[1] != k0 or Q0[l].stride(0) != 1:
            raise ValueError("Q0 must be column-major float64 n_l x k0")
        q[l] = Q0[l].data_ptr()
        ld[l] = max(Q0[l].stride(1), Q0[l].shape[0])
    need = int(L.rhosvd_c2t_start_workspace_size(_c.byref(cp), _c.byref(opts), k0))
    if need == 0:
        raise RhosvdError(RHOSVD_ERR_INVALID_ARG, "rhosvd_c2t_start_workspace_size")
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=U[0].device)
    if out is None:
        out = alloc_tucker([cp.n[l] for l in range(3)], cp.R, r_max, U[0].device, with_V, with_xi)
    t = tucker_struct(out)
    rc = L.rhosvd_c2t_start(_c.byref(cp), _c.byref(opts), q, ld, k0, int(iters), _c.byref(t),
                            _c.c_void_p(workspace.data_ptr()), _c.c_size_t(workspace.numel()), _stream_handle(stream))
    if rc != RHOSVD_OK:
        raise RhosvdError(rc, "rhosvd_c2t_start")
    return out


class Mlp:
    """The proposal network (device weights owned by the library handle)."""

    IN, OUT = 128, 2048

    def __init__(self, batch_max=256, seed=0):
        L = load()
        h = _c.c_void_p()
        rc = L.rhosvd_mlp_create(int(batch_max), int(seed) & 0xFFFFFFFFFFFFFFFF, _c.byref(h))
        if rc != RHOSVD_OK:
            raise RhosvdError(rc, "rhosvd_mlp_create")
        self.h = h
        self.batch_max = int(batch_max)

    def close(self):
        if self.h:
            load().rhosvd_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forward(self, X, stream=None):
        torch = _torch()
        B = X.shape[0]
        Y = torch.empty(B, self.OUT, dtype=torch.float32, device=X.device)
        rc = load().rhosvd_mlp_forward(self.h, _c.c_void_p(X.data_ptr()), B, _c.c_void_p(Y.data_ptr()),
                                       _stream_handle(stream))
        if rc != RHOSVD_OK:
            raise RhosvdError(rc, "rhosvd_mlp_forward")
        return Y

    def gradients(self, X, G, stream=None):
        torch = _torch()
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
        rc = load().rhosvd_mlp_gradients(self.h, _c.c_void_p(X.data_ptr()), _c.c_void_p(G.data_ptr()), X.shape[0],
                                         _c.c_void_p(loss.data_ptr()), _stream_handle(stream))
        if rc != RHOSVD_OK:
            raise RhosvdError(rc, "rhosvd_mlp_gradients")
        return loss

    def train_step(self, X, G, lr, stream=None):
        torch = _torch()
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
        rc = load().rhosvd_mlp_train_step(self.h, _c.c_void_p(X.data_ptr()), _c.c_void_p(G.data_ptr()), X.shape[0],
                                          _c.c_float(lr), _c.c_void_p(loss.data_ptr()), _stream_handle(stream))
        if rc != RHOSVD_OK:
            raise RhosvdError(rc, "rhosvd_mlp_train_step")
        return loss

    def params(self, which=0):
        """All parameters (which=0) or the last gradients (which=1) as one float32 numpy vector."""
        import numpy as np
        buf = np.empty(int(load().rhosvd_mlp_num_params()), dtype=np.float32)
        rc = load().rhosvd_mlp_params(self.h, _c.c_void_p(buf.ctypes.data), 1, int(which))
        if rc != RHOSVD_OK:
            raise RhosvdError(rc, "rhosvd_mlp_params")
        return buf

    def set_params(self, vec):
        import numpy as np
        buf = np.ascontiguousarray(vec, dtype=np.float32)
        rc = load().rhosvd_mlp_params(self.h, _c.c_void_p(buf.ctypes.data), 0, 0)
        if rc != RHOSVD_OK:
            raise RhosvdError(rc, "rhosvd_mlp_params")

    def save(self, path):
        """Checkpoint: weights, Adam moments and step count into one binary file."""
        rc = load().rhosvd_mlp_save(self.h, os.fsencode(path))
        if rc != RHOSVD_OK:
            raise RhosvdError(rc, "rhosvd_mlp_save")

    def load_state(self, path):
        """Resume from a checkpoint written by save() (the handle is unchanged on error)."""
        rc = load().rhosvd_mlp_load(self.h, os.fsencode(path))
        if rc != RHOSVD_OK:
            raise RhosvdError(rc, "rhosvd_mlp_load")

    def status(self, stream=None):
        """Raise if a tensor-core product of the network hit its bounded wait since the last check."""
        rc = load().rhosvd_mlp_status(self.h, _stream_handle(stream))
        if rc != RHOSVD_OK:
            raise RhosvdError(rc, "rhosvd_mlp_status")


def rhosvd_probe_fp64(blocks, iters, out, stream=None):
    """Launch the FP64 fma-rate probe (4096 * iters FLOP a block) writing into `out`
    (float64 CUDA tensor of blocks * 256 entries)."""
    if out.dtype != _torch().float64 or out.numel() < blocks * 256 or not out.is_cuda:
        raise ValueError("out must be a float64 CUDA tensor of blocks * 256 entries")
    rc = load().rhosvd_probe_fp64(int(blocks), int(iters), _c.c_void_p(out.data_ptr()), _stream_handle(stream))
    if rc != RHOSVD_OK:
        raise RhosvdError(rc, "rhosvd_probe_fp64")


def rhosvd_features(centres, loga, c, cbox, la, lb, stream=None):
    """(3, 128) float32 features of one Gaussian sum (device float64 inputs)."""
    torch = _torch()
    out = torch.empty(3, 128, dtype=torch.float32, device=centres.device)
    rc = load().rhosvd_features(_c.c_void_p(centres.data_ptr()), _c.c_void_p(loga.data_ptr()),
                                _c.c_void_p(c.data_ptr()), int(c.numel()), float(cbox), float(la), float(lb),
                                _c.c_void_p(out.data_ptr()), _stream_handle(stream))
    if rc != RHOSVD_OK:
        raise RhosvdError(rc, "rhosvd_features")
    return out


def rhosvd_chebyshev(n, b, device="cuda", stream=None):
    """Q_T: n x 64 column-major float64 (orthonormal discrete Chebyshev basis of the grid)."""
    torch = _torch()
    T = torch.empty(64, n, dtype=torch.float64, device=device)
    rc = load().rhosvd_chebyshev(int(n), float(b), _c.c_void_p(T.data_ptr()), _stream_handle(stream))
    if rc != RHOSVD_OK:
        raise RhosvdError(rc, "rhosvd_chebyshev")
    return T.t()


def rhosvd_proj_target(QT, Z, r, stream=None):
    """G (64 x 64 float32, G[i + 64 i']) of the leading r columns of Z (column-major)."""
    torch = _torch()
    G = torch.empty(64 * 64, dtype=torch.float32, device=Z.device)
    ldz = max(Z.stride(1), Z.shape[0])
    rc = load().rhosvd_proj_target(int(QT.shape[0]), _c.c_void_p(QT.data_ptr()), _c.c_void_p(Z.data_ptr()), ldz,
                                   int(r), _c.c_void_p(G.data_ptr()), _stream_handle(stream))
    if rc != RHOSVD_OK:
        raise RhosvdError(rc, "rhosvd_proj_target")
    return G


def rhosvd_proposal_basis(QT, Y, stream=None):
    """Q0 (n x 32 column-major float64) from one mode's network output Y (2048 float32)."""
    torch = _torch()
    n = int(QT.shape[0])
    Q0 = torch.empty(32, n, dtype=torch.float64, device=Y.device)
    rc = load().rhosvd_proposal_basis(n, _c.c_void_p(QT.data_ptr()), _c.c_void_p(Y.data_ptr()),
                                      _c.c_void_p(Q0.data_ptr()), _stream_handle(stream))
    if rc != RHOSVD_OK:
        raise RhosvdError(rc, "rhosvd_proposal_basis")
    return Q0.t()

