"""Host logic of the batched rank grid search (no GPU: a fake server stands in
for the library and 'completes' each job with an error that depends on its
ranks, so the selection can be checked)."""
import numpy as np
import pytest

from paper_2511_16358_gb300 import rank_search as rs


class FakeServer:
    """Records the call order; the completed tensor of a job is the truth plus
    a deterministic perturbation whose size is |R_{0,1} - 6| + |R_{0,2} - 3|
    (so the best point of a grid is known) plus a floor."""
    FP64, OK = 0, 0

    def __init__(self, xt):
        self.xt = xt
        self.calls = []
        self.jobs = {}
        self.destroyed = 0
        self.fail_poll = False

    def tensor_dtype(self, precision):
        return np.float64

    def make_problem(self, dims, R, **kw):
        return {"dims": dims, "R": np.array(R), **kw}

    def server_create(self, budget, slots):
        self.calls.append("create")
        return object()

    def submit(self, srv, prob, obs, mask, init):
        t = len(self.jobs) + 1
        self.jobs[t] = (prob, mask.copy())
        self.calls.append("submit")
        return t

    def poll(self, srv, t, out, timeout_us=-1):
        self.calls.append("poll")
        if self.fail_poll:
            raise RuntimeError("device failure")
        prob, _ = self.jobs[t]
        R = prob["R"]
        err = abs(int(R[0, 1]) - 6) + abs(int(R[0, 2]) - 3) + 0.5
        pert = np.cos(np.arange(self.xt.size)).reshape(self.xt.shape)
        out[...] = self.xt + 1e-3 * err * pert
        return self.OK, {"sweeps_done": 10, "converged": 1}

    def server_destroy(self, srv):
        self.destroyed += 1


def _data(shape=(6, 5, 4), p=0.5):
    rng = np.random.default_rng(3)
    xt = rng.random(shape)
    mask = (rng.random(shape) < p).astype(np.uint8)
    return xt, mask


def test_msi_grid_is_the_papers_grid():
    full = rs.msi_grid()
    assert len(full) == 18
    assert all(R[0, 2] == R[1, 2] == R[2, 0] == R[2, 1] for R in full)
    assert sorted({int(R[0, 1]) for R in full}) == [3, 6, 9, 15, 30, 36]
    for R in full:
        rs.check_ranks(3, R)  # every point is within the library's order-3 limits
    capped = rs.msi_grid(max_rank=6)
    assert [(int(R[0, 1]), int(R[0, 2])) for R in capped] == [(3, 3), (3, 6), (6, 3), (6, 6)]


def test_rank_limits_follow_the_order():
    rs.check_ranks(3, rs.rank_matrix(3, {(0, 1): 64, (0, 2): 64, (1, 2): 1}))
    with pytest.raises(ValueError):
        rs.check_ranks(3, rs.rank_matrix(3, {(0, 1): 65, (0, 2): 2, (1, 2): 2}))
    with pytest.raises(ValueError):  # Q_0 = 64 * 65 > 4096
        rs.check_ranks(3, rs.rank_matrix(3, {(0, 1): 64, (0, 2): 65, (1, 2): 1}))
    with pytest.raises(ValueError):
        rs.check_ranks(4, rs.rank_matrix(4, {(0, 1): 9, (0, 2): 2, (0, 3): 2, (1, 2): 2, (1, 3): 2, (2, 3): 2}))


def test_edge_grid_enumerates_every_combination():
    g = rs.edge_grid(4, {(0, 1): [2, 5], (2, 3): [3, 4, 6], "default": [2]})
    assert len(g) == 6
    seen = {(int(R[0, 1]), int(R[2, 3])) for R in g}
    assert seen == {(a, c) for a in (2, 5) for c in (3, 4, 6)}
    for R in g:
        assert (R == R.T).all() and R[0, 2] == R[1, 3] == 2


def test_holdout_split_partitions_the_observed_set():
    _, mask = _data((40, 30, 20), 0.3)
    fit, held = rs.holdout_split(mask, 0.2, seed=7)
    obs = mask.astype(bool)
    assert not (fit.astype(bool) & held).any()
    assert ((fit.astype(bool) | held) == obs).all()
    assert abs(held.sum() / obs.sum() - 0.2) < 0.02
    fit2, held2 = rs.holdout_split(mask, 0.2, seed=7)
    assert (held2 == held).all()


@pytest.mark.parametrize("with_truth", [True, False])
def test_search_batches_all_jobs_and_picks_the_best_point(with_truth):
    xt, mask = _data()
    fake = FakeServer(xt)
    grid = rs.edge_grid(3, {(0, 1): [3, 6, 8], (0, 2): [3, 5], "default": [2]})
    res = rs.search(xt * mask, mask, grid, xtrue=xt if with_truth else None, holdout=0.25,
                    backend=fake)
    # all jobs are queued before the first result is awaited, and the server is released
    assert fake.calls == ["create"] + ["submit"] * len(grid) + ["poll"] * len(grid)
    assert fake.destroyed == 1
    assert res.criterion == ("rse" if with_truth else "holdout")
    assert (int(res.best_ranks[0, 1]), int(res.best_ranks[0, 2])) == (6, 3)
    assert res.best_index == int(np.argmin(res.scores))
    # without truth, the jobs never see the held-out entries
    if not with_truth:
        for _, m in fake.jobs.values():
            assert m.sum() < mask.sum()
    else:
        for _, m in fake.jobs.values():
            assert (m == mask).all()


def test_ties_go_to_fewer_parameters():
    xt, mask = _data()

    class Flat(FakeServer):
        def poll(self, srv, t, out, timeout_us=-1):
            out[...] = self.xt
            return self.OK, {}

    grid = [rs.rank_matrix(3, {(0, 1): r, (0, 2): 2, (1, 2): 2}) for r in (5, 2, 4)]
    res = rs.search(xt * mask, mask, grid, xtrue=xt, backend=Flat(xt))
    assert int(res.best_ranks[0, 1]) == 2
    assert res.params[1] == rs.param_count(xt.shape, grid[1]) == 6 * 4 + 5 * 4 + 4 * 4


def test_server_released_when_a_job_fails_and_bad_grids_refused():
    xt, mask = _data()
    fake = FakeServer(xt)
    fake.fail_poll = True
    with pytest.raises(RuntimeError):
        rs.search(xt * mask, mask, rs.msi_grid(), xtrue=xt, backend=fake)
    assert fake.destroyed == 1
    with pytest.raises(ValueError):
        rs.search(xt * mask, mask, [], xtrue=xt, backend=FakeServer(xt))
    with pytest.raises(ValueError):
        rs.search(xt * mask, mask, [rs.rank_matrix(3, {(0, 1): 65, (0, 2): 3, (1, 2): 3})], xtrue=xt,
                  backend=FakeServer(xt))
    with pytest.raises(ValueError):
        rs.search(xt * mask, mask, rs.msi_grid(), holdout=0.0, backend=FakeServer(xt))
