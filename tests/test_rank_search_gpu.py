"""The batched rank grid search (Sec. 5, 5.2) on the GPU: every grid point is a
completion job on one server, all queued at once.  Each job's score equals
the FP64 oracle's completion of the same problem from the same seeded start,
and the search picks the oracle's best point.  Both scoring criteria run:
RSE against the ground truth, and the error on held-out observed entries."""
import numpy as np
import pytest

import oracle
from paper_2511_16358_gb300 import binding as b
from paper_2511_16358_gb300 import rank_search as rs
from tests._cases import make_case, scaled_uniform_start

pytestmark = pytest.mark.gpu

DIMS = (20, 18, 12)
SWEEPS = 20
SEED = 77


def _grid():
    return rs.edge_grid(3, {(0, 1): [2, 3, 4], (0, 2): [2, 3], (1, 2): [2]})


def _oracle_scores(case, grid, fit_mask, score):
    out = []
    for R in grid:
        X0 = oracle.init_x(case["xt"], fit_mask)
        G = scaled_uniform_start(DIMS, R, X0, fit_mask, SEED)
        X = X0.copy()
        oracle.complete(DIMS, R, 0.1, G, X, fit_mask, max_sweeps=SWEEPS, tol=0.0)
        out.append(score(X))
    return out


def test_rank_search_rse_scores_match_oracle():
    case = make_case(DIMS, {(0, 1): 3, (0, 2): 2, (1, 2): 2}, 0.4, seed=481, kind="max1", sigma=0.02)
    xt, mask = case["xt"], case["mask"]
    grid = _grid()
    res = rs.search(xt * mask, mask, grid, rho=0.1, max_sweeps=SWEEPS, tol=0.0, precision=b.FP64, xtrue=xt,
                    seed=SEED, hbm_budget_bytes=8 << 30, slots=4)
    den = np.linalg.norm(xt)
    want = _oracle_scores(case, grid, mask, lambda X: float(np.linalg.norm(xt - X) / den))
    np.testing.assert_allclose(res.scores, want, rtol=1e-9)
    assert res.best_index == int(np.argmin(want))
    assert all(st["sweeps_done"] == SWEEPS for st in res.stats)


def test_rank_search_holdout_scores_match_oracle():
    case = make_case(DIMS, {(0, 1): 3, (0, 2): 2, (1, 2): 2}, 0.5, seed=482, kind="max1", sigma=0.02)
    xt, mask = case["xt"], case["mask"]
    obs = xt * mask
    grid = _grid()
    res = rs.search(obs, mask, grid, rho=0.1, max_sweeps=SWEEPS, tol=0.0, precision=b.FP64, holdout=0.2,
                    seed=SEED, hbm_budget_bytes=8 << 30, slots=3)
    fit, held = rs.holdout_split(mask, 0.2, SEED)
    ref = obs[held]
    want = _oracle_scores(dict(case, xt=obs), grid, fit,
                          lambda X: float(np.linalg.norm(X[held] - ref) / np.linalg.norm(ref)))
    np.testing.assert_allclose(res.scores, want, rtol=1e-9)
    assert res.best_index == int(np.argmin(want))


def test_rank_search_over_ranks_above_eight_matches_oracle():
    """Points of the multispectral grid with R_{1,2} in {15, 36} (Sec. 5.2) next
    to small ones, all on one server: each score equals the oracle's."""
    case = make_case(DIMS, {(0, 1): 3, (0, 2): 2, (1, 2): 2}, 0.4, seed=483, kind="max1", sigma=0.02)
    xt, mask = case["xt"], case["mask"]
    grid = [R for R in rs.edge_grid(3, {(0, 1): [3, 15, 36], (0, 2): [3, 9], (1, 2): [3, 9]})
            if R[0, 2] == R[1, 2]]
    res = rs.search(xt * mask, mask, grid, rho=0.1, max_sweeps=SWEEPS, tol=0.0, precision=b.FP64, xtrue=xt,
                    seed=SEED, hbm_budget_bytes=8 << 30, slots=4)
    den = np.linalg.norm(xt)
    want = _oracle_scores(case, grid, mask, lambda X: float(np.linalg.norm(xt - X) / den))
    np.testing.assert_allclose(res.scores, want, rtol=1e-9)
    assert res.best_index == int(np.argmin(want))
