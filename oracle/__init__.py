"""FP64 CPU oracle of iFCTN tensor completion -- TEST INFRASTRUCTURE ONLY.

This package is the independent checker of the GPU library.  Only the test
suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import it.  It shares no code with the CUDA path: the arithmetic lives in
``ifctn_oracle.c`` (plain C, FP64, compensated sums) and this module only
builds that file with gcc and marshals numpy arrays into it.

Functions follow the paper's notation (Gan & Cui, iFCTN):
  reconstruct     eq. (iFCTN), Def. 2
  pair_matrix     W_{p,q} = G_{p,q}^T G_{q,p}, the factors of S_k in Prop. 1
  block_system    A_j^T A_j and A_j^T x_j of eq. (updateG) for one column
  sweep           one pass of Algorithm 1: eq. (updateG) for every block in
                  Gauss-Seidel order, then eq. (updateX)
  complete        Algorithm 1 until the relative-change test or t_max
  init_x          X^0 = P_Omega(O)
  objective       f(G, X) = 1/2 ||X - iFCTN(G)||_F^2 (Sec. 4.1)
  param_count     sum_k I_k sum_{l != k} R_{k,l} (Sec. 4.3, Table 5)

Layout: C-order tensors; factor block G_{k,l} is R_{k,l} x I_k row-major,
packed by k then l != k; ranks as a 4x4 row-major int matrix.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ifctn_oracle.c")
_LIB = os.path.join(_HERE, "libifctn_oracle.so")
_lock = threading.Lock()
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_dp = ctypes.POINTER(ctypes.c_double)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available) and return the .so path."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off", "-fno-fast-math"]
    tmp = _LIB + f".tmp{os.getpid()}"
    try:
        subprocess.run(base + ["-fopenmp", _SRC, "-o", tmp, "-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + [_SRC, "-o", tmp, "-lm"], check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.ifo_numel.restype = ctypes.c_longlong
            lib.ifo_factor_offset.restype = ctypes.c_longlong
            lib.ifo_param_count.restype = ctypes.c_longlong
            lib.ifo_objective.restype = ctypes.c_double
            for name in ("ifo_reconstruct", "ifo_block_system", "ifo_sweep", "ifo_complete",
                         "ifo_cholesky_solve"):
                getattr(lib, name).restype = ctypes.c_int
            _lib = lib
    return _lib


def _shape_args(dims, ranks):
    dims = np.ascontiguousarray(np.asarray(dims, dtype=np.int64))
    R = np.zeros((4, 4), dtype=np.int32)
    rk = np.asarray(ranks, dtype=np.int32)
    R[: rk.shape[0], : rk.shape[1]] = rk
    R = np.ascontiguousarray(R)
    return len(dims), dims, R


def _p(a, t):
    return a.ctypes.data_as(t)


def factor_offset(dims, ranks, k, l):
    N, d, R = _shape_args(dims, ranks)
    return int(_load().ifo_factor_offset(N, _p(d, _i64p), _p(R, _i32p), k, l))


def param_count(dims, ranks):
    N, d, R = _shape_args(dims, ranks)
    return int(_load().ifo_param_count(N, _p(d, _i64p), _p(R, _i32p)))


def pair_matrix(dims, ranks, G, p, q):
    N, d, R = _shape_args(dims, ranks)
    G = np.ascontiguousarray(G, dtype=np.float64)
    W = np.empty((d[p], d[q]), dtype=np.float64)
    _load().ifo_pair_matrix(N, _p(d, _i64p), _p(R, _i32p), _p(G, _dp), p, q, _p(W, _dp))
    return W


def reconstruct(dims, ranks, G):
    N, d, R = _shape_args(dims, ranks)
    G = np.ascontiguousarray(G, dtype=np.float64)
    out = np.empty(tuple(int(x) for x in d), dtype=np.float64)
    rc = _load().ifo_reconstruct(N, _p(d, _i64p), _p(R, _i32p), _p(G, _dp), _p(out, _dp))
    if rc:
        raise RuntimeError(f"ifo_reconstruct failed ({rc})")
    return out


def block_system(dims, ranks, G, X, k, i, j):
    """H = A_j^T A_j and b = A_j^T x_j for column j of G_{k,i} (no proximal terms)."""
    N, d, R = _shape_args(dims, ranks)
    G = np.ascontiguousarray(G, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    n = int(R[k, i])
    H = np.zeros((n, n), dtype=np.float64)
    b = np.zeros(n, dtype=np.float64)
    rc = _load().ifo_block_system(N, _p(d, _i64p), _p(R, _i32p), _p(G, _dp), _p(X, _dp),
                                  k, i, ctypes.c_longlong(j), _p(H, _dp), _p(b, _dp))
    if rc:
        raise RuntimeError(f"ifo_block_system failed ({rc})")
    return H, b


def init_x(O, mask):
    O = np.ascontiguousarray(O, dtype=np.float64)
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    X = np.empty_like(O)
    _load().ifo_init_x(ctypes.c_longlong(O.size), _p(O, _dp), _p(m, _u8p), _p(X, _dp))
    return X


def objective(dims, ranks, G, X):
    N, d, R = _shape_args(dims, ranks)
    G = np.ascontiguousarray(G, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    return float(_load().ifo_objective(N, _p(d, _i64p), _p(R, _i32p), _p(G, _dp), _p(X, _dp)))


STAT_KEYS = ("rel_change", "objective", "rse", "rmse", "dx2", "x2")


def sweep(dims, ranks, rho, G, X, mask, xtrue=None, nthreads=0):
    """One PAM sweep in place on (G, X).  Returns the stats dict."""
    N, d, R = _shape_args(dims, ranks)
    assert G.dtype == np.float64 and G.flags.c_contiguous
    assert X.dtype == np.float64 and X.flags.c_contiguous
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    xt = None if xtrue is None else np.ascontiguousarray(xtrue, dtype=np.float64)
    st = np.zeros(6, dtype=np.float64)
    rc = _load().ifo_sweep(N, _p(d, _i64p), _p(R, _i32p), ctypes.c_double(rho), _p(G, _dp),
                           _p(X, _dp), _p(m, _u8p), None if xt is None else _p(xt, _dp),
                           int(nthreads), _p(st, _dp))
    if rc < 0:
        raise RuntimeError(f"ifo_sweep failed ({rc})")
    if rc > 0:
        raise FloatingPointError("non-SPD normal equations in ifo_sweep")
    return dict(zip(STAT_KEYS, st.tolist()))


def complete(dims, ranks, rho, G, X, mask, max_sweeps, tol=0.0, xtrue=None, nthreads=0):
    """Algorithm 1 in place on (G, X).  Returns a list of per-sweep stats dicts."""
    N, d, R = _shape_args(dims, ranks)
    assert G.dtype == np.float64 and G.flags.c_contiguous
    assert X.dtype == np.float64 and X.flags.c_contiguous
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    xt = None if xtrue is None else np.ascontiguousarray(xtrue, dtype=np.float64)
    log = np.zeros((max(max_sweeps, 1), 6), dtype=np.float64)
    done = ctypes.c_int(0)
    rc = _load().ifo_complete(N, _p(d, _i64p), _p(R, _i32p), ctypes.c_double(rho),
                              int(max_sweeps), ctypes.c_double(tol), _p(G, _dp), _p(X, _dp),
                              _p(m, _u8p), None if xt is None else _p(xt, _dp), int(nthreads),
                              _p(log, _dp), ctypes.byref(done))
    if rc < 0:
        raise RuntimeError(f"ifo_complete failed ({rc})")
    return [dict(zip(STAT_KEYS, row.tolist())) for row in log[: done.value]]


def cholesky_solve(H, rhs):
    H = np.array(H, dtype=np.float64, order="C")
    x = np.array(rhs, dtype=np.float64)
    rc = _load().ifo_cholesky_solve(int(H.shape[0]), _p(H, _dp), _p(x, _dp))
    if rc:
        raise FloatingPointError("non-positive pivot")
    return x


def omp_threads_available() -> int:
    return os.cpu_count() or 1


def metrics(xtrue, X, mask):
    """(RSE, RMSE) of Sec. 5: RSE = ||Xt-X||/||Xt||, RMSE over the missing entries."""
    xt = np.ascontiguousarray(xtrue, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    out = np.zeros(2, dtype=np.float64)
    _load().ifo_metrics(ctypes.c_longlong(xt.size), _p(xt, _dp), _p(X, _dp), _p(m, _u8p),
                        _p(out, _dp))
    return float(out[0]), float(out[1])
