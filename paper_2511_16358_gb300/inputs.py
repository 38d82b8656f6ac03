"""Seeded synthetic inputs for iFCTN tensor completion.

This module is the only piece shared by the GPU path's tests/benchmark and the
CPU oracle's tests.  It holds random draws and their post-processing only --
none of the method's arithmetic.  The planted tensor itself (iFCTN of the
drawn factors) is computed by whichever side consumes the factors.

Generator: splitmix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) used as a counter-based stream: draw n of
stream ``seed`` is mix(seed + (n+1) * 0x9E3779B97F4A7C15).  Uniforms take the
top 53 bits; normals use Box-Muller on consecutive uniform pairs.

Workloads are shaped after the paper's experiments (Sec. 5): multispectral
images 256x256x31, colour video, traffic tensors, the synthetic 20^4 Tucker
tensor; the datasets themselves are not used.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Draws offset..offset+n-1 of the counter-based splitmix64 stream ``seed``."""
    with np.errstate(over="ignore"):
        ctr = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + ctr * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, n: int) -> np.ndarray:
    """U[0,1) doubles from the top 53 bits."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, n: int) -> np.ndarray:
    """N(0,1) doubles by Box-Muller on uniform pairs."""
    m = (n + 1) // 2
    u = uniform(seed, 2 * m).reshape(m, 2)
    rad = np.sqrt(-2.0 * np.log1p(-u[:, 0]))
    ang = 2.0 * np.pi * u[:, 1]
    return np.stack([rad * np.cos(ang), rad * np.sin(ang)], axis=1).reshape(-1)[:n]


# ---------------------------------------------------------------------------
# problem shapes and factor packing (the convention of the C ABI)
# ---------------------------------------------------------------------------

def rank_matrix(N: int, edge_ranks) -> np.ndarray:
    """4x4 symmetric rank matrix from a dict {(k,l): R} (k<l) or a scalar."""
    R = np.zeros((4, 4), dtype=np.int32)
    for k in range(N):
        for l in range(k + 1, N):
            r = edge_ranks if np.isscalar(edge_ranks) else edge_ranks[(k, l)]
            R[k, l] = R[l, k] = int(r)
    return R


def factor_blocks(dims, R):
    """[(k, l, rows, cols, offset)] for the packed factor array: G_{k,l} is
    R_{k,l} x I_k row-major, packed by k then l != k."""
    N = len(dims)
    out, off = [], 0
    for k in range(N):
        for l in range(N):
            if l == k:
                continue
            n = int(R[k][l]) * int(dims[k])
            out.append((k, l, int(R[k][l]), int(dims[k]), off))
            off += n
    return out


def factor_size(dims, R) -> int:
    b = factor_blocks(dims, R)
    return b[-1][4] + b[-1][2] * b[-1][3]


def unpack_factors(G, dims, R):
    """dict (k,l) -> view of G_{k,l} (R_{k,l} x I_k)."""
    return {(k, l): G[off:off + r * c].reshape(r, c) for k, l, r, c, off in factor_blocks(dims, R)}


def gaussian_factors(dims, R, seed: int) -> np.ndarray:
    """Every cherry factor entry i.i.d. N(0,1), packed."""
    return normal(seed, factor_size(dims, R))


def uniform_factors(dims, R, seed: int, lo=0.0, hi=1.0) -> np.ndarray:
    return lo + (hi - lo) * uniform(seed, factor_size(dims, R))


# ---------------------------------------------------------------------------
# masks and noise
# ---------------------------------------------------------------------------

def uniform_mask(shape, p_observed: float, seed: int) -> np.ndarray:
    """Bernoulli(p) observation mask, one uint8 per entry (1 = observed)."""
    n = int(np.prod(shape))
    return (uniform(seed, n) < p_observed).astype(np.uint8).reshape(shape)


def fiber_mask(shape, fiber_mode: int, fiber_missing: float, p_observed: float, seed: int):
    """Structured mask: a fraction ``fiber_missing`` of the mode-``fiber_mode``
    fibers is unobserved entirely; elsewhere entries are observed w.p. p."""
    shape = tuple(int(s) for s in shape)
    rest = [s for m, s in enumerate(shape) if m != fiber_mode]
    nf = int(np.prod(rest))
    drop = uniform(seed + 1, nf) < fiber_missing
    m = uniform_mask(shape, p_observed, seed)
    drop_full = np.expand_dims(drop.reshape(rest), axis=fiber_mode)
    m = np.where(np.broadcast_to(drop_full, shape), 0, m).astype(np.uint8)
    return m


def tucker_tensor(dims, core_ranks, seed: int) -> np.ndarray:
    """Tucker-generated tensor of the paper's synthetic experiment (Sec. 5.1).

    Core C (r_1 x ... x r_N) and factor matrices U_k (I_k x r_k) have i.i.d.
    U(0,1) entries, drawn in that order from the one stream ``seed``; the
    tensor is C x_1 U_1 x_2 U_2 ... x_N U_N (mode-k products), divided by its
    largest entry so that it lies in [0, 1] (the experiments pre-normalise
    every dataset to [0, 1]).  Its multilinear rank is (r_1, ..., r_N).  This
    is data preparation: the completion model is iFCTN, not Tucker.
    """
    dims = tuple(int(d) for d in dims)
    core_ranks = tuple(int(r) for r in core_ranks)
    ncore = int(np.prod(core_ranks))
    u = uniform(seed, ncore + sum(d * r for d, r in zip(dims, core_ranks)))
    T = u[:ncore].reshape(core_ranks)
    off = ncore
    for k, (d, r) in enumerate(zip(dims, core_ranks)):
        U = u[off:off + d * r].reshape(d, r)
        off += d * r
        # mode-k product: contract mode k of T with the columns of U, keep the axis order
        T = np.moveaxis(np.tensordot(U, T, axes=([1], [k])), 0, k)
    return np.ascontiguousarray(T / T.max())


def gaussian_noise(shape, sigma: float, seed: int) -> np.ndarray:
    return sigma * normal(seed, int(np.prod(shape))).reshape(shape)


def finalize(planted: np.ndarray, kind: str, noise=None) -> np.ndarray:
    """Value-range post-processing of a planted tensor (data preparation only).

    'max1'     : scale so max|x| = 1
    'minmax01' : affine map to [0,1], add noise, clip to [0,1]
    'abs01'    : |x| scaled to [0,1], add noise, clip at 0
    """
    x = np.asarray(planted, dtype=np.float64)
    if kind == "max1":
        y = x / np.max(np.abs(x))
        return y if noise is None else y + noise
    if kind == "minmax01":
        lo, hi = float(x.min()), float(x.max())
        y = (x - lo) / (hi - lo)
        if noise is not None:
            y = y + noise
        return np.clip(y, 0.0, 1.0)
    if kind == "abs01":
        y = np.abs(x)
        y = y / y.max()
        if noise is not None:
            y = y + noise
        return np.maximum(y, 0.0)
    raise ValueError(kind)


# ---------------------------------------------------------------------------
# named workloads (shapes of the paper's experiments)
# ---------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    dims: tuple
    R: np.ndarray
    rho: float
    sweeps: int
    p_observed: float
    kind: str
    sigma: float
    precision: str
    seed_base: int
    fiber: tuple | None = None          # (mode, fraction) for fiber-missing masks
    extra: dict = field(default_factory=dict)
    tucker: tuple | None = None         # core ranks: the truth is Tucker-generated, not planted iFCTN

    @property
    def planted(self) -> bool:
        """True when the truth is an iFCTN tensor of Gaussian factors, which the
        consumer computes (oracle or library) and passes to workload_inputs."""
        return self.tucker is None

    @property
    def N(self):
        return len(self.dims)


def _video_ranks():
    R = rank_matrix(4, {(0, 1): 8, (0, 3): 8, (1, 3): 8, (0, 2): 3, (1, 2): 3, (2, 3): 3})
    return R


WORKLOADS = {
    # planted order-3 30^3, all R=3, 30% observed, rho 0.1, 50 sweeps, FP64
    "cube30_r3": Workload("cube30_r3", (30, 30, 30), rank_matrix(3, 3), 0.1, 50, 0.30,
                          "max1", 0.0, "fp64", 1),
    # multispectral-image shaped 256x256x31, R=6, 10% observed, noise 0.01, 100 sweeps
    "msi256x256x31_r6": Workload("msi256x256x31_r6", (256, 256, 31), rank_matrix(3, 6), 0.1,
                                 100, 0.10, "minmax01", 0.01, "mixed", 2),
    # colour-video shaped 144x176x3x100, R=8 spatial/temporal, 3 on colour edges, 5% observed
    "video144x176x3x100": Workload("video144x176x3x100", (144, 176, 3, 100), _video_ranks(),
                                   0.1, 100, 0.05, "minmax01", 0.02, "mixed", 3),
    # traffic shaped 288x400x60x24, R=5, 5% observed + 20% of mode-2 fibers missing
    "traffic288x400x60x24_r5": Workload("traffic288x400x60x24_r5", (288, 400, 60, 24),
                                        rank_matrix(4, 5), 0.1, 200, 0.05, "abs01", 0.05,
                                        "mixed", 5, fiber=(1, 0.20)),
    # the paper's synthetic experiment shape (Sec. 5.1): 20^4
    "synthetic20x4": Workload("synthetic20x4", (20, 20, 20, 20), rank_matrix(4, 5), 0.1, 1000,
                              0.2, "raw", 0.0, "fp64", 6),
}

# The paper's synthetic experiment (Sec. 5.1, Fig. 3): a 20^4 tensor of Tucker rank
# (5,5,5,5) with U(0,1) core and factors, completed at random-missing rates up to 90%
# with the experiments' defaults (rho = 0.1, t_max = 1000, eps = 1e-5).  The text gives
# no iFCTN rank for it; every R_{k,l} = 5 (the Tucker rank) is the reading taken.
TUCKER_MISSING_RATES = (0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9)
for _m in TUCKER_MISSING_RATES:
    _name = f"tucker20x4_rm{int(round(100 * _m)):02d}"
    WORKLOADS[_name] = Workload(_name, (20, 20, 20, 20), rank_matrix(4, 5), 0.1, 1000,
                                round(1.0 - _m, 10), "raw", 0.0, "fp64", 7,
                                extra={"tol": 1e-5}, tucker=(5, 5, 5, 5))


def workload_inputs(w: Workload, planted: np.ndarray | None):
    """Given the planted tensor (computed by the caller from
    ``gaussian_factors(w.dims, w.R, 1000 + w.seed_base)``; None for a workload
    whose truth is Tucker-generated), return (X_true, mask, G0) for the
    workload."""
    shape = w.dims
    if w.tucker is not None:
        planted = tucker_tensor(shape, w.tucker, 1000 + w.seed_base)
    noise = gaussian_noise(shape, w.sigma, 3000 + w.seed_base) if w.sigma > 0 else None
    xt = planted if w.kind == "raw" else finalize(planted, w.kind, noise)
    if w.fiber is not None:
        mask = fiber_mask(shape, w.fiber[0], w.fiber[1], w.p_observed, 2000 + w.seed_base)
    else:
        mask = uniform_mask(shape, w.p_observed, 2000 + w.seed_base)
    G0 = uniform_factors(w.dims, w.R, 4000 + w.seed_base)
    return xt, mask, G0


def planted_factor_seed(w: Workload) -> int:
    return 1000 + w.seed_base
