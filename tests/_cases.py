"""Seeded test cases shared by the parity tests (inputs only; planted tensors
and scalings come from the oracle, never from the GPU path)."""
import contextlib
import os

import numpy as np

import oracle
from paper_2511_16358_gb300 import inputs as inp


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (den if den > 0 else 1.0))


def scaled_uniform_start(dims, R, xobs, mask, seed):
    """U(0,1) factors rescaled by one common factor so that
    ||iFCTN(G0)|| = ||P_Omega(O)|| / sqrt(p) (computed with the oracle)."""
    G0 = inp.uniform_factors(dims, R, seed)
    rec = oracle.reconstruct(dims, R, G0)
    nobs = max(int(mask.sum()), 1)
    target = np.linalg.norm(xobs) * np.sqrt(mask.size / nobs)
    ratio = target / max(np.linalg.norm(rec), 1e-300)
    N = len(dims)
    return G0 * ratio ** (1.0 / (N * (N - 1)))


def make_case(dims, edge, p_obs, seed, kind="max1", sigma=0.0, fiber=None):
    """Planted iFCTN tensor (Gaussian factors) -> X_true, mask, G0, X0."""
    N = len(dims)
    R = inp.rank_matrix(N, edge)
    Gt = inp.gaussian_factors(dims, R, 1000 + seed)
    planted = oracle.reconstruct(dims, R, Gt)
    noise = inp.gaussian_noise(dims, sigma, 3000 + seed) if sigma > 0 else None
    xt = inp.finalize(planted, kind, noise) if kind != "raw" else planted
    if fiber is not None:
        mask = inp.fiber_mask(dims, fiber[0], fiber[1], p_obs, 2000 + seed)
    else:
        mask = inp.uniform_mask(dims, p_obs, 2000 + seed)
    X0 = oracle.init_x(xt, mask)
    G0 = scaled_uniform_start(dims, R, X0, mask, 4000 + seed)
    return dict(dims=tuple(dims), R=R, Gtrue=Gt, xt=xt, mask=mask, G0=G0, X0=X0)


@contextlib.contextmanager
def path(name):
    """Forces the execution path of contexts created inside the block:
    "persistent" (one cooperative launch per call, the default for tensors that
    stay in L2) or "graph" (per-stage kernels with the warp-pipelined
    contraction, the default for HBM-sized tensors)."""
    old = os.environ.get("IFCTN_PATH")
    os.environ["IFCTN_PATH"] = name
    try:
        yield
    finally:
        if old is None:
            del os.environ["IFCTN_PATH"]
        else:
            os.environ["IFCTN_PATH"] = old
