"""Plain CPU FP64 oracle for RHOSVD (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  The compute lives in ``rhosvd_oracle.c`` (plain C, FP64,
explicit loops); this module compiles it with gcc on first use and marshals numpy
arrays through ctypes.  It shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rhosvd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "librhosvd_oracle.so")
_lock = threading.Lock()
_lib = None

ORC_OK, ORC_ERR_ARG, ORC_ERR_NOMEM, ORC_ERR_NOTCONV, ORC_ERR_RANK = 0, -1, -2, -3, -4


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, -O2, no FMA contraction so x86 and Arm agree)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c99",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            dpp = ctypes.POINTER(dp)
            L.orc_col_norm.restype = ctypes.c_double
            L.orc_col_norm.argtypes = [ctypes.c_int, dp]
            L.orc_householder_r.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, dp]
            L.orc_jacobi_left.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, ctypes.c_int]
            L.orc_side_svd.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, ctypes.c_int]
            L.orc_eps_rank.argtypes = [ctypes.c_int, dp, ctypes.c_double]
            L.orc_normalize.argtypes = [ip, ctypes.c_int, dpp, ip, dp, dpp, dp, dp, ip]
            L.orc_project.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp]
            L.orc_project.restype = None
            L.orc_core.argtypes = [ctypes.c_int, ip, dp, dp, dp, dp, dp]
            L.orc_core.restype = None
            L.orc_c2t.argtypes = [ip, ctypes.c_int, dpp, ip, dp, ctypes.c_double, ip, ctypes.c_int,
                                  ctypes.c_int, ip, dpp, dpp, dpp, dp, dp, dp]
            L.orc_cp_hadamard.argtypes = [ip, ctypes.c_int, dpp, dp, ctypes.c_int, dpp, dp, dpp, dp]
            L.orc_cp_hadamard.restype = None
            L.orc_cp_sum.argtypes = [ip, ctypes.c_double, ctypes.c_int, dpp, dp, ctypes.c_double,
                                     ctypes.c_int, dpp, dp, dpp, dp]
            L.orc_cp_sum.restype = None
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _dpp(arrs):
    return (ctypes.POINTER(ctypes.c_double) * len(arrs))(*[_dp(a) for a in arrs])


def _f64(a):
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def col_norm(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    return lib().orc_col_norm(x.shape[0], _dp(x))


def householder_r(A):
    """R factor (n x n) of the Householder QR of A (m x n, m >= n)."""
    A = _f64(A).copy(order="F")
    m, n = A.shape
    Rf = np.zeros((n, n), order="F")
    rc = lib().orc_householder_r(m, n, _dp(A), m, _dp(Rf))
    if rc != 0:
        raise RuntimeError(f"orc_householder_r failed: {rc}")
    return Rf


def jacobi_left(A, max_sweeps=100):
    """One-sided Jacobi: (sigma descending, Z) with A = Z diag(sigma) V^T."""
    A = _f64(A).copy(order="F")
    m, n = A.shape
    sig = np.zeros(n)
    Z = np.zeros((m, n), order="F")
    rc = lib().orc_jacobi_left(m, n, _dp(A), _dp(sig), _dp(Z), max_sweeps)
    if rc < 0:
        raise RuntimeError(f"orc_jacobi_left failed: {rc}")
    return sig, Z


def side_svd(Un, max_sweeps=100):
    """(sigma, Z) of a side matrix (n x R), q = min(n, R) values/vectors."""
    Un = _f64(Un)
    n, R = Un.shape
    q = min(n, R)
    sig = np.zeros(q)
    Z = np.zeros((n, q), order="F")
    rc = lib().orc_side_svd(n, R, _dp(Un), _dp(sig), _dp(Z), max_sweeps)
    if rc < 0:
        raise RuntimeError(f"orc_side_svd failed: {rc}")
    return sig, Z


def eps_rank(sigma, eps):
    s = np.ascontiguousarray(sigma, dtype=np.float64)
    return int(lib().orc_eps_rank(s.shape[0], _dp(s), float(eps)))


def normalize(U, xi):
    """(Un list, xin, norms (3,R), keep) per the normalisation rule of the oracle."""
    U = [_f64(u) for u in U]
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    R = xi.shape[0]
    n = np.array([u.shape[0] for u in U], dtype=np.int32)
    ld = n.copy()
    Un = [np.zeros((int(n[l]), R), order="F") for l in range(3)]
    xin = np.zeros(R)
    norms = np.zeros(3 * R)
    keep = np.zeros(R, dtype=np.int32)
    lib().orc_normalize(_ip(n), R, _dpp(U), _ip(ld), _dp(xi), _dpp(Un), _dp(xin), _dp(norms), _ip(keep))
    return Un, xin, norms.reshape(3, R), keep


def project(Z, Un):
    """V = Z^T Un (r x R) by the oracle's explicit loops (Prop. 2.2: D_{l,0} V_0^T = Z_0^T U)."""
    Z = _f64(Z)
    Un = _f64(Un)
    n, r = Z.shape
    R = Un.shape[1]
    V = np.zeros((r, R), order="F")
    lib().orc_project(n, R, r, _dp(Z), _dp(Un), _dp(V))
    return V


def core(V, xin):
    """beta(i, j, m) = sum_nu xin_nu V1(i, nu) V2(j, nu) V3(m, nu) by the oracle's explicit
    loops (Prop. 2.2); returns an (r1, r2, r3) array."""
    V = [_f64(v) for v in V]
    xin = np.ascontiguousarray(xin, dtype=np.float64)
    r = np.array([v.shape[0] for v in V], dtype=np.int32)
    R = xin.shape[0]
    beta = np.zeros(max(int(np.prod(r)), 1))
    lib().orc_core(R, _ip(r), _dp(V[0]), _dp(V[1]), _dp(V[2]), _dp(xin), _dp(beta))
    return beta[: int(np.prod(r))].reshape(tuple(int(x) for x in r), order="F")


def c2t(U, xi, eps=1e-6, ranks=(0, 0, 0), r_max=None, max_sweeps=100):
    """The whole RHOSVD.  Returns a dict with Z (list of n_l x r_l), beta (r1,r2,r3 array,
    index [i,j,m]), sigma (list), V (list of r_l x R), xin, ranks, kept, xi_norm, tails."""
    U = [_f64(u) for u in U]
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    R = xi.shape[0]
    n = np.array([u.shape[0] for u in U], dtype=np.int32)
    ld = n.copy()
    q = [min(int(n[l]), R) for l in range(3)]
    if r_max is None:
        r_max = max(max(q), 1)
    Z = [np.zeros((int(n[l]), max(q[l], 1)), order="F") for l in range(3)]
    sig = [np.zeros(max(q[l], 1)) for l in range(3)]
    V = [np.zeros(max(r_max * R, 1)) for _ in range(3)]
    beta = np.zeros(max(r_max ** 3, 1))
    xin = np.zeros(max(R, 1))
    stats = np.zeros(4)
    rr = np.zeros(3, dtype=np.int32)
    rk = np.asarray(ranks, dtype=np.int32)
    rc = lib().orc_c2t(_ip(n), R, _dpp(U), _ip(ld), _dp(xi), float(eps), _ip(rk), int(r_max),
                       int(max_sweeps), _ip(rr), _dpp(Z), _dpp(sig), _dpp(V), _dp(beta), _dp(xin),
                       _dp(stats))
    if rc != 0:
        raise RuntimeError(f"orc_c2t failed: {rc} (ranks {rr.tolist()})")
    r = [int(x) for x in rr]
    out = dict(ranks=r, kept=int(stats[0]), xi_norm=float(stats[1]), xin=xin[:R].copy())
    out["Z"] = [np.asfortranarray(Z[l][:, : r[l]]) for l in range(3)]
    out["Z_full"] = [Z[l][:, : q[l]] for l in range(3)]
    out["sigma"] = [sig[l][: q[l]].copy() for l in range(3)]
    out["V"] = [V[l][: r[l] * R].reshape((r[l], R), order="F") for l in range(3)]
    out["beta"] = beta[: r[0] * r[1] * r[2]].reshape((r[0], r[1], r[2]), order="F")
    out["tails"] = [float(np.sqrt(np.sum(out["sigma"][l][r[l]:] ** 2))) for l in range(3)]
    return out


def c2t_threads(U, xi, eps=1e-6, ranks=(0, 0, 0), max_sweeps=100):
    """The same RHOSVD as ``c2t`` (the steps of orc_c2t in its order: normalisation, per mode
    the full side-matrix SVD and its eps-rank, V = Z^T U~, the core), with the three modes'
    SVDs run at once in three host threads (ctypes releases the GIL during each C call; the
    C routines keep no global state).  Returns the same dict, plus the wall time of each step."""
    import time
    from concurrent.futures import ThreadPoolExecutor
    t0 = time.perf_counter()
    Un, xin, _, keep = normalize(U, xi)
    t1 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=3) as ex:
        svd = list(ex.map(lambda l: side_svd(Un[l], max_sweeps), range(3)))
    t2 = time.perf_counter()
    r = []
    for l in range(3):
        sig = svd[l][0]
        q = sig.shape[0]
        r.append(min(ranks[l], q) if ranks[l] > 0 else eps_rank(sig, eps))
    Z = [np.asfortranarray(svd[l][1][:, : r[l]]) for l in range(3)]
    V = [project(Z[l], Un[l]) for l in range(3)]
    t3 = time.perf_counter()
    beta = core(V, xin)
    t4 = time.perf_counter()
    out = dict(ranks=r, kept=int(keep.sum()), xi_norm=float(np.sqrt(np.sum(xin * xin))), xin=xin,
               Z=Z, Z_full=[svd[l][1] for l in range(3)], sigma=[svd[l][0] for l in range(3)], V=V, beta=beta)
    out["tails"] = [float(np.sqrt(np.sum(out["sigma"][l][r[l]:] ** 2))) for l in range(3)]
    out["seconds"] = dict(normalize=t1 - t0, svd=t2 - t1, project=t3 - t2, core=t4 - t3)
    return out


def cp_hadamard(Ua, xa, Ub, xb):
    Ua = [_f64(u) for u in Ua]
    Ub = [_f64(u) for u in Ub]
    xa = np.ascontiguousarray(xa, dtype=np.float64)
    xb = np.ascontiguousarray(xb, dtype=np.float64)
    Ra, Rb = xa.shape[0], xb.shape[0]
    n = np.array([u.shape[0] for u in Ua], dtype=np.int32)
    Uc = [np.zeros((int(n[l]), Ra * Rb), order="F") for l in range(3)]
    xc = np.zeros(Ra * Rb)
    lib().orc_cp_hadamard(_ip(n), Ra, _dpp(Ua), _dp(xa), Rb, _dpp(Ub), _dp(xb), _dpp(Uc), _dp(xc))
    return Uc, xc


def cp_sum(alpha, Ua, xa, beta, Ub, xb):
    Ua = [_f64(u) for u in Ua]
    Ub = [_f64(u) for u in Ub]
    xa = np.ascontiguousarray(xa, dtype=np.float64)
    xb = np.ascontiguousarray(xb, dtype=np.float64)
    Ra, Rb = xa.shape[0], xb.shape[0]
    n = np.array([u.shape[0] for u in Ua], dtype=np.int32)
    Uc = [np.zeros((int(n[l]), Ra + Rb), order="F") for l in range(3)]
    xc = np.zeros(Ra + Rb)
    lib().orc_cp_sum(_ip(n), float(alpha), Ra, _dpp(Ua), _dp(xa), float(beta), Rb, _dpp(Ub), _dp(xb),
                     _dpp(Uc), _dp(xc))
    return Uc, xc
