"""Batched iFCTN-rank grid search on the completion server.

The experiments choose the iFCTN ranks R_{k,l} per dataset from a grid and
report the best result, and the times they report include that tuning
(Sec. 5; the multispectral grid is R_{1,2} in {3,6,9,15,30,36},
R_{1,3} = R_{2,3} in {3,6,9}, Sec. 5.2).  Every grid point is an independent
completion job, so the search submits all of them to one server at once; the
server's continuous batching keeps as many resident as slots and the device
budget allow and overlaps their kernels.  The completions run in the
library's kernels; this module only builds the jobs, splits the mask and
scores the returned tensors.

Command line (one GPU): ``python -m paper_2511_16358_gb300.rank_search
--workload msi256x256x31_r6`` searches the multispectral grid on that
workload and prints one JSON line (scores, best ranks, wall time of the whole
search).

Scoring:
  * with a ground truth (the experiments' protocol, synthetic data):
    RSE = ||X_true - X|| / ||X_true|| of each completed tensor;
  * without one: a seeded share of the observed entries is held out of every
    job, and the score is the relative error on those held-out entries.
The lowest score wins; ties go to the point with fewer parameters
(sum_k I_k sum_{l != k} R_{k,l}), then to the earlier grid point.
"""
from __future__ import annotations

import argparse
import json
import time
from dataclasses import dataclass, field

import numpy as np

# per-edge rank limits of the library: 8 in general (the register-resident
# stage kernels), 64 for order-3 tensors with every Q_k = prod_{l != k} R_{k,l}
# at most 4096 (the chain kernels for wide ranks)
MAX_EDGE_RANK = 8
MAX_EDGE_RANK_ORDER3 = 64
MAX_Q_ORDER3 = 4096


def check_ranks(N: int, R) -> None:
    """Raises ValueError when the library would refuse rank matrix R."""
    lim = MAX_EDGE_RANK_ORDER3 if N == 3 else MAX_EDGE_RANK
    for k in range(N):
        for l in range(N):
            if k != l and not 1 <= int(R[k][l]) <= lim:
                raise ValueError(f"edge rank R[{k},{l}] = {int(R[k][l])} outside 1..{lim}")
    if N == 3:
        for k in range(N):
            q = int(np.prod([int(R[k][l]) for l in range(N) if l != k]))
            if q > MAX_Q_ORDER3:
                raise ValueError(f"Q_{k} = {q} above {MAX_Q_ORDER3}")


def rank_matrix(N: int, edges: dict) -> np.ndarray:
    """4x4 symmetric rank matrix from {(k, l): R_{k,l}} over the pairs k < l."""
    R = np.zeros((4, 4), dtype=np.int32)
    for (k, l), r in edges.items():
        R[k, l] = R[l, k] = int(r)
    return R


def msi_grid(max_rank: int = 36) -> list:
    """The multispectral grid of Sec. 5.2 for an order-3 tensor (18 points),
    without the points that need an edge rank above ``max_rank``."""
    out = []
    for r12 in (3, 6, 9, 15, 30, 36):
        for r13 in (3, 6, 9):
            if max(r12, r13) <= max_rank:
                out.append(rank_matrix(3, {(0, 1): r12, (0, 2): r13, (1, 2): r13}))
    return out


def edge_grid(N: int, choices: dict) -> list:
    """Every combination of per-edge choices {(k, l): [R, ...]}, pairs k < l;
    edges not named take the first value of ``choices['default']``."""
    pairs = [(k, l) for k in range(N) for l in range(k + 1, N)]
    lists = [list(choices.get(p, choices.get("default", [1]))) for p in pairs]
    out = []
    for combo in np.array(np.meshgrid(*lists, indexing="ij")).reshape(len(pairs), -1).T:
        out.append(rank_matrix(N, dict(zip(pairs, combo.tolist()))))
    return out


def param_count(dims, R) -> int:
    """Number of iFCTN parameters, sum_k I_k sum_{l != k} R_{k,l} (Sec. 4.3)."""
    N = len(dims)
    return int(sum(int(dims[k]) * int(R[k][l]) for k in range(N) for l in range(N) if l != k))


def holdout_split(mask, fraction: float, seed: int):
    """Splits the observed set into (fit mask as uint8, held-out boolean mask)
    by a seeded Bernoulli(fraction) draw per observed entry."""
    obs = np.asarray(mask).astype(bool)
    draw = np.random.default_rng(seed).random(obs.shape) < fraction
    held = obs & draw
    return (obs & ~held).astype(np.uint8), held


@dataclass
class SearchResult:
    criterion: str                 # "rse" (against a ground truth) or "holdout"
    grid: list                     # the rank matrices searched, in submission order
    scores: list                   # one score per grid point (lower is better)
    stats: list                    # the server's per-job stats (sweeps_done, converged, ...)
    best_index: int
    best_ranks: np.ndarray
    best_x: np.ndarray             # completed tensor of the best point
    seconds: float                 # wall time of the whole search (submit to last result)
    params: list = field(default_factory=list)


def search(obs, mask, grid, *, rho=0.1, max_sweeps=1000, tol=1e-5, precision=None, xtrue=None,
           holdout=0.1, seed=0, hbm_budget_bytes=100 << 30, slots=16, backend=None) -> SearchResult:
    """Completes ``obs`` (observed where ``mask`` is 1) once per rank matrix of
    ``grid`` on one server and returns the best point (see module docstring).

    ``backend`` defaults to the library binding; it must provide the binding's
    server_create / submit / poll / server_destroy / make_problem /
    tensor_dtype and its FP64 and OK constants.
    """
    if backend is None:
        from paper_2511_16358_gb300 import binding as backend
    b = backend
    if not grid:
        raise ValueError("empty rank grid")
    precision = b.FP64 if precision is None else precision
    dims = tuple(int(d) for d in np.shape(obs))
    for R in grid:
        check_ranks(len(dims), R)
    dt = b.tensor_dtype(precision)
    obs_h = np.ascontiguousarray(obs, dtype=dt)
    if xtrue is None:
        if not 0.0 < holdout < 1.0:
            raise ValueError("holdout must lie in (0, 1) when no ground truth is given")
        fit_mask, held = holdout_split(mask, holdout, seed)
        if not held.any():
            raise ValueError("no observed entry was held out")
        criterion = "holdout"
    else:
        fit_mask, held = np.ascontiguousarray(mask, dtype=np.uint8), None
        criterion = "rse"

    if criterion == "rse":
        xt = np.asarray(xtrue, dtype=np.float64)
        den = np.linalg.norm(xt)

        def score(X):
            return float(np.linalg.norm(xt - X.astype(np.float64)) / den)
    else:
        ref = np.asarray(obs, dtype=np.float64)[held]
        den = np.linalg.norm(ref)

        def score(X):
            return float(np.linalg.norm(X.astype(np.float64)[held] - ref) / den)

    params = [param_count(dims, R) for R in grid]
    t0 = time.perf_counter()
    srv = b.server_create(int(hbm_budget_bytes), int(slots))
    scores, stats, best, best_x = [], [], None, None
    try:
        # every job is queued before the first result is awaited: the server
        # batches them as slots and budget allow
        tickets = [b.submit(srv, b.make_problem(dims, R, rho=rho, max_sweeps=max_sweeps, tol=tol,
                                                precision=precision, seed=seed),
                            obs_h, fit_mask, None) for R in grid]
        for n, t in enumerate(tickets):
            out = np.empty(dims, dtype=dt)
            rc, st = b.poll(srv, t, out, timeout_us=-1)
            if rc != b.OK:
                raise RuntimeError(f"rank-search job {t} ended with status {rc}")
            stats.append(st)
            scores.append(score(out))
            # only the best completed tensor so far is kept
            if best is None or (scores[n], params[n]) < (scores[best], params[best]):
                best, best_x = n, out
    finally:
        b.server_destroy(srv)
    seconds = time.perf_counter() - t0
    return SearchResult(criterion, list(grid), scores, stats, best, np.asarray(grid[best]), best_x,
                        seconds, params)


def _planted(b, inp, w):
    """The workload's truth: iFCTN of its Gaussian factors, reconstructed by
    the library (None for a Tucker-generated truth, which inputs builds)."""
    if not w.planted:
        return None
    dims = w.dims
    Gt = inp.gaussian_factors(dims, w.R, inp.planted_factor_seed(w))
    P = int(np.prod(dims))
    ctx = b.create(b.make_problem(dims, w.R, rho=w.rho, max_sweeps=0, tol=0.0, precision=b.FP64),
                   np.zeros(P), np.zeros(P, dtype=np.uint8), Gt)
    try:
        return b.reconstruct(ctx, np.empty(dims, dtype=np.float64))
    finally:
        b.destroy(ctx)


def main(argv=None):
    ap = argparse.ArgumentParser(description="batched iFCTN-rank grid search on one GPU")
    ap.add_argument("--workload", default="msi256x256x31_r6")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--sweeps", type=int, default=None, help="t_max per job (default: the workload's)")
    ap.add_argument("--tol", type=float, default=1e-5)
    ap.add_argument("--criterion", default="rse", choices=["rse", "holdout"])
    ap.add_argument("--slots", type=int, default=16)
    args = ap.parse_args(argv)

    import __graft_entry__
    __graft_entry__.build()
    from . import binding as b
    from . import inputs as inp

    w = inp.WORKLOADS[args.workload]
    N = len(w.dims)
    xt, mask, _ = inp.workload_inputs(w, _planted(b, inp, w))
    grid = msi_grid() if N == 3 else [rank_matrix(N, {(k, l): r for k in range(N) for l in range(k + 1, N)})
                                      for r in (3, 5, 8)]
    prec = b.MIXED if args.precision == "mixed" else b.FP64
    res = search(xt * mask, mask, grid, rho=w.rho, max_sweeps=args.sweeps or w.sweeps, tol=args.tol,
                 precision=prec, xtrue=xt if args.criterion == "rse" else None, slots=args.slots)

    def edges(R):
        return {f"R{k + 1}{l + 1}": int(R[k][l]) for k in range(N) for l in range(k + 1, N)}

    print(json.dumps({
        "workload": w.name, "criterion": res.criterion, "precision": args.precision,
        "points": [dict(edges(R), score=sc, sweeps=st.get("sweeps_done"), params=pc)
                   for R, sc, st, pc in zip(res.grid, res.scores, res.stats, res.params)],
        "best": dict(edges(res.best_ranks), score=res.scores[res.best_index]),
        "seconds_including_tuning": res.seconds}), flush=True)


if __name__ == "__main__":
    main()

