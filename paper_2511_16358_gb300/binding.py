"""ctypes binding of libifctn.so -- argument marshalling only.

Every function mirrors an entry point of include/ifctn.h with the same name
(minus the ``ifctn_`` prefix).  Arrays may be numpy arrays (host memory) or
torch tensors (host or CUDA memory); they are passed by pointer, never copied
here.  All computation runs in the library's CUDA kernels; there is no CPU
fallback: loading fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libifctn.so")

FP64 = 0
MIXED = 1

OK, EINVAL, ENOMEM, ECUDA, ENOTSPD, EBUSY, ENOTREADY, ETIMEOUT, ENOTFOUND = range(9)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ENOTSPD", "EBUSY", "ENOTREADY", "ETIMEOUT",
                "ENOTFOUND"]

EXPORTED = [
    "ifctn_create", "ifctn_sweep", "ifctn_complete", "ifctn_reconstruct", "ifctn_get_factors",
    "ifctn_set_factors", "ifctn_get_x", "ifctn_set_x", "ifctn_set_truth", "ifctn_get_log",
    "ifctn_mode_system", "ifctn_kernels_per_sweep", "ifctn_destroy", "ifctn_server_create",
    "ifctn_submit", "ifctn_poll", "ifctn_server_info_get", "ifctn_server_latency",
    "ifctn_server_destroy", "ifctn_last_error", "ifctn_sweep_async", "ifctn_launch_stage",
    "ifctn_launch_count", "ifctn_phase_times", "ifctn_reconstruct_noalloc", "ifctn_wait_selftest",
    "ifctn_tune", "ifctn_tune_choose", "ifctn_sweep_exchange",
]


class Problem(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int32), ("dims", ctypes.c_int64 * 4), ("ranks", ctypes.c_int32 * 16),
                ("rho", ctypes.c_double), ("max_sweeps", ctypes.c_int32), ("tol", ctypes.c_double),
                ("precision", ctypes.c_int32), ("seed", ctypes.c_uint64)]


class Stats(ctypes.Structure):
    _fields_ = [("sweeps_done", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("rel_change", ctypes.c_double), ("objective", ctypes.c_double),
                ("rse", ctypes.c_double), ("rmse", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ServerInfo(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int64), ("resident", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("bytes_in_use", ctypes.c_int64), ("peak_resident", ctypes.c_int64),
                ("batch_launches", ctypes.c_int64), ("batched_jobs", ctypes.c_int64)]


# int32_t (*)(void* user, double* values, int64_t count)
ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int64)


class IfctnError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


_lib = None


def load(path: str | None = None):
    """Load libifctn.so (built by ``_build.build``).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"libifctn.so not built ({p}); run __graft_entry__.build()")
    lib = ctypes.CDLL(p)
    vp, i32, i64, u64, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    P = ctypes.POINTER
    sig = {
        "ifctn_create": (i32, [P(Problem), vp, vp, vp, vp, P(vp)]),
        "ifctn_sweep": (i32, [vp, i32, P(Stats)]),
        "ifctn_complete": (i32, [vp, vp, P(Stats)]),
        "ifctn_reconstruct": (i32, [vp, vp]),
        "ifctn_get_factors": (i32, [vp, vp]),
        "ifctn_set_factors": (i32, [vp, vp]),
        "ifctn_get_x": (i32, [vp, vp]),
        "ifctn_set_x": (i32, [vp, vp]),
        "ifctn_set_truth": (i32, [vp, vp, i32]),
        "ifctn_get_log": (i32, [vp, P(Stats), i32, P(i32)]),
        "ifctn_mode_system": (i32, [vp, i32, vp, vp]),
        "ifctn_kernels_per_sweep": (i32, [vp]),
        "ifctn_destroy": (None, [vp]),
        "ifctn_server_create": (i32, [ctypes.c_size_t, i32, P(vp)]),
        "ifctn_submit": (i32, [vp, P(Problem), vp, vp, vp, P(u64)]),
        "ifctn_poll": (i32, [vp, u64, vp, P(Stats), i64]),
        "ifctn_server_info_get": (i32, [vp, P(ServerInfo)]),
        "ifctn_server_latency": (i32, [vp, u64, P(dp)]),
        "ifctn_server_destroy": (None, [vp]),
        "ifctn_last_error": (ctypes.c_char_p, []),
        "ifctn_sweep_async": (i32, [vp, i32]),
        "ifctn_launch_stage": (i32, [vp, i32, i32]),
        "ifctn_launch_count": (i64, [vp]),
        "ifctn_phase_times": (i32, [vp, P(dp), i32, P(i32)]),
        "ifctn_reconstruct_noalloc": (i32, [i32, P(i64), P(i32), i32, vp, vp, vp]),
        "ifctn_wait_selftest": (i32, [vp, i64]),
        "ifctn_tune": (i32, [vp, ctypes.c_char_p, P(i32)]),
        "ifctn_tune_choose": (i32, [i32, P(dp)]),
        "ifctn_sweep_exchange": (i32, [vp, i32, ALLREDUCE_FN, vp, P(Stats)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def last_error() -> str:
    return load().ifctn_last_error().decode()


def _check(rc):
    if rc != OK:
        raise IfctnError(rc, last_error())


def ptr(a):
    """Raw pointer of a numpy array or torch tensor (host or device); None passes NULL."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("arrays passed to the library must be C-contiguous (np.ascontiguousarray)")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors passed to the library must be contiguous (.contiguous())")
        return a.data_ptr()
    raise TypeError(type(a))


def make_problem(dims, ranks, rho=0.1, max_sweeps=1000, tol=1e-5, precision=FP64, seed=0) -> Problem:
    p = Problem()
    p.order = len(dims)
    for k, d in enumerate(dims):
        p.dims[k] = int(d)
    R = np.asarray(ranks)
    for k in range(R.shape[0]):
        for l in range(R.shape[1]):
            p.ranks[k * 4 + l] = int(R[k, l])
    p.rho = float(rho)
    p.max_sweeps = int(max_sweeps)
    p.tol = float(tol)
    p.precision = int(precision)
    p.seed = int(seed)
    return p


def tensor_dtype(precision):
    return np.float64 if precision == FP64 else np.float32


# ---------------------------------------------------------------------------
# context entry points
# ---------------------------------------------------------------------------

def create(prob: Problem, obs, mask, init_factors=None, stream=None):
    ctx = ctypes.c_void_p()
    _check(load().ifctn_create(ctypes.byref(prob), ptr(obs), ptr(mask), ptr(init_factors), stream,
                               ctypes.byref(ctx)))
    return ctx


def sweep(ctx, n=1) -> dict:
    st = Stats()
    _check(load().ifctn_sweep(ctx, int(n), ctypes.byref(st)))
    return st.as_dict()


def sweep_async(ctx, n=1):
    _check(load().ifctn_sweep_async(ctx, int(n)))


def launch_stage(ctx, stage, k=0):
    _check(load().ifctn_launch_stage(ctx, int(stage), int(k)))


def complete(ctx, out_X=None) -> dict:
    st = Stats()
    _check(load().ifctn_complete(ctx, ptr(out_X), ctypes.byref(st)))
    return st.as_dict()


def reconstruct(ctx, out):
    _check(load().ifctn_reconstruct(ctx, ptr(out)))
    return out


def get_factors(ctx, out):
    _check(load().ifctn_get_factors(ctx, ptr(out)))
    return out


def set_factors(ctx, G):
    _check(load().ifctn_set_factors(ctx, ptr(G)))


def get_x(ctx, out):
    _check(load().ifctn_get_x(ctx, ptr(out)))
    return out


def set_x(ctx, X):
    _check(load().ifctn_set_x(ctx, ptr(X)))


def set_truth(ctx, xtrue, log=True):
    _check(load().ifctn_set_truth(ctx, ptr(xtrue), 1 if log else 0))


def get_log(ctx, max_n=4096) -> list:
    arr = (Stats * max_n)()
    n = ctypes.c_int32(0)
    _check(load().ifctn_get_log(ctx, arr, int(max_n), ctypes.byref(n)))
    return [arr[i].as_dict() for i in range(n.value)]


def mode_system(ctx, k, Mk, Kk):
    _check(load().ifctn_mode_system(ctx, int(k), ptr(Mk), ptr(Kk)))
    return Mk, Kk


def wait_selftest(ctx, budget_cycles):
    """Runs the library's bounded device waits on conditions nothing satisfies;
    returns the status (IFCTN_ETIMEOUT when the waits expired as designed)."""
    return int(load().ifctn_wait_selftest(ctx, int(budget_cycles)))


def sweep_exchange(ctx, n, allreduce) -> dict:
    """n sweeps of a slab context (ifctn_sweep_exchange); ``allreduce(values)``
    receives a float64 numpy view of host memory and must replace it in place
    by the sum over the processes (the same bits everywhere)."""
    err = []

    def cb(_user, ptr_, count):
        try:
            allreduce(np.ctypeslib.as_array(ptr_, shape=(int(count),)))
            return 0
        except Exception as e:  # reported after the call returns
            err.append(e)
            return 1

    fn = ALLREDUCE_FN(cb)
    st = Stats()
    rc = load().ifctn_sweep_exchange(ctx, int(n), fn, None, ctypes.byref(st))
    if err:
        raise err[0]
    _check(rc)
    return st.as_dict()


def tune(ctx, cache_path=None) -> int:
    """Autotunes the streaming contraction's launch shapes (cache_path: the
    tuning cache file, or None); returns the number of candidate plans timed."""
    n = ctypes.c_int32(0)
    _check(load().ifctn_tune(ctx, None if cache_path is None else str(cache_path).encode(), ctypes.byref(n)))
    return n.value


def tune_choose(seconds) -> int:
    """The tuner's selection rule on a list of timings (default first)."""
    a = (ctypes.c_double * max(len(seconds), 1))(*[float(x) for x in seconds])
    return int(load().ifctn_tune_choose(len(seconds), a))


def kernels_per_sweep(ctx) -> int:
    return int(load().ifctn_kernels_per_sweep(ctx))


def launch_count(ctx) -> int:
    return int(load().ifctn_launch_count(ctx))


def phase_times(ctx) -> list:
    arr = (ctypes.c_double * 64)()
    n = ctypes.c_int32(0)
    _check(load().ifctn_phase_times(ctx, arr, 64, ctypes.byref(n)))
    return [arr[i] for i in range(n.value)]


def _noalloc_check(name, t, dtype_name, numel):
    """The C entry point receives no buffer lengths, so the binding checks
    every buffer it passes: a torch tensor of the right dtype and size,
    contiguous, in CUDA memory of the current device (a short or mistyped
    buffer would be read or written past its end on the GPU)."""
    if not hasattr(t, "data_ptr"):
        raise ValueError(f"{name} must be a CUDA torch tensor, got {type(t).__name__}")
    if str(t.dtype) != f"torch.{dtype_name}":
        raise ValueError(f"{name} must be {dtype_name}, got {t.dtype}")
    if t.numel() != numel:
        raise ValueError(f"{name} must hold {numel} elements, got {t.numel()}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _noalloc_device_check(name, t):
    if not t.is_cuda:
        raise ValueError(f"{name} must be in CUDA memory of the current device")
    import torch
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is "
                         f"cuda:{torch.cuda.current_device()}")


def reconstruct_noalloc(dims, ranks, precision, factors_dev, out_dev, stream=None):
    """Allocation-free reconstruction: factors_dev / out_dev are CUDA tensors
    of the current device (factors FP64, out in the precision's tensor dtype);
    nothing is allocated by the library."""
    R = np.asarray(ranks)
    N = len(dims)
    nfac = sum(int(R[k, l]) * int(dims[k]) for k in range(N) for l in range(N) if l != k)
    _noalloc_check("factors_dev", factors_dev, "float64", nfac)
    _noalloc_check("out_dev", out_dev, "float64" if precision == FP64 else "float32",
                   int(np.prod([int(x) for x in dims])))
    _noalloc_device_check("factors_dev", factors_dev)
    _noalloc_device_check("out_dev", out_dev)
    d = (ctypes.c_int64 * 4)(*([int(x) for x in dims] + [0] * (4 - len(dims))))
    r = (ctypes.c_int32 * 16)()
    for k in range(R.shape[0]):
        for l in range(R.shape[1]):
            r[k * 4 + l] = int(R[k, l])
    _check(load().ifctn_reconstruct_noalloc(len(dims), d, r, int(precision), ptr(factors_dev), ptr(out_dev),
                                            stream))
    return out_dev


def destroy(ctx):
    if ctx:
        load().ifctn_destroy(ctx)


# ---------------------------------------------------------------------------
# serving entry points
# ---------------------------------------------------------------------------

def server_create(hbm_budget_bytes: int, max_slots: int):
    s = ctypes.c_void_p()
    _check(load().ifctn_server_create(int(hbm_budget_bytes), int(max_slots), ctypes.byref(s)))
    return s


def submit(srv, prob: Problem, obs, mask, init_factors=None) -> int:
    t = ctypes.c_uint64(0)
    _check(load().ifctn_submit(srv, ctypes.byref(prob), ptr(obs), ptr(mask), ptr(init_factors),
                               ctypes.byref(t)))
    return t.value


def poll(srv, ticket, out_X=None, timeout_us=-1):
    """Returns (status, stats dict).  Raises on failures other than not-ready/timeout."""
    st = Stats()
    rc = load().ifctn_poll(srv, ctypes.c_uint64(ticket), ptr(out_X), ctypes.byref(st), int(timeout_us))
    if rc in (ENOTREADY, ETIMEOUT):
        return rc, None
    _check(rc)
    return rc, st.as_dict()


def server_info_get(srv) -> dict:
    i = ServerInfo()
    _check(load().ifctn_server_info_get(srv, ctypes.byref(i)))
    return {f: getattr(i, f) for f, _ in i._fields_}


def server_latency(srv, ticket) -> float:
    v = ctypes.c_double(0)
    _check(load().ifctn_server_latency(srv, ctypes.c_uint64(ticket), ctypes.byref(v)))
    return v.value


def server_destroy(srv):
    if srv:
        load().ifctn_server_destroy(srv)


class Completion:
    """Owns one context: Algorithm 1 on one tensor."""

    def __init__(self, dims, ranks, obs, mask, rho=0.1, max_sweeps=1000, tol=1e-5, precision=FP64,
                 init_factors=None, seed=0, stream=None):
        self.dims = tuple(int(d) for d in dims)
        self.ranks = np.asarray(ranks)
        self.precision = precision
        self.prob = make_problem(dims, ranks, rho, max_sweeps, tol, precision, seed)
        self.ctx = create(self.prob, obs, mask, init_factors, stream)

    @property
    def dtype(self):
        return tensor_dtype(self.precision)

    def nfactors(self):
        N = len(self.dims)
        return sum(int(self.ranks[k, l]) * self.dims[k] for k in range(N) for l in range(N) if l != k)

    def sweep(self, n=1):
        return sweep(self.ctx, n)

    def complete(self, out_X=None):
        return complete(self.ctx, out_X)

    def factors(self):
        return get_factors(self.ctx, np.empty(self.nfactors(), dtype=np.float64))

    def set_factors(self, G):
        set_factors(self.ctx, np.ascontiguousarray(G, dtype=np.float64))

    def x(self):
        return get_x(self.ctx, np.empty(self.dims, dtype=self.dtype))

    def set_x(self, X):
        set_x(self.ctx, np.ascontiguousarray(X, dtype=self.dtype))

    def reconstruct(self):
        return reconstruct(self.ctx, np.empty(self.dims, dtype=self.dtype))

    def close(self):
        destroy(self.ctx)
        self.ctx = None

    def __del__(self):
        try:
            if self.ctx:
                self.close()
        except Exception:
            pass
