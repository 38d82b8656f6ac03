"""The seeded input generators and workload recipes (CPU).

The generator is checked against the published splitmix64 outputs for seed 0
(the reference implementation of Steele, Lea & Flood's generator, as
distributed with xoroshiro), the derived uniforms and normals by their
moments, and each workload recipe against the shapes, ranks, value ranges and
observation patterns of the paper's experiments (Sec. 5).
"""
import numpy as np
import pytest

import oracle
from paper_2511_16358_gb300 import inputs as inp


def test_splitmix64_matches_published_outputs_for_seed_zero():
    got = [int(v) for v in inp.splitmix64(0, 3)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    # the counter form: draw n of a stream is independent of how many are taken
    assert int(inp.splitmix64(0, 1, offset=2)[0]) == got[2]


def test_uniform_and_normal_moments():
    u = inp.uniform(12345, 1_000_000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 2e-3 and abs(u.var() - 1 / 12) < 1e-3
    z = inp.normal(12345, 1_000_001)
    assert z.size == 1_000_001
    assert abs(z.mean()) < 5e-3 and abs(z.var() - 1.0) < 5e-3
    assert abs(np.mean(z ** 4) - 3.0) < 0.05


def test_fiber_mask_drops_whole_fibers_and_samples_the_rest():
    shape = (30, 40, 12, 10)
    m = inp.fiber_mask(shape, 1, 0.2, 0.05, seed=9)
    fibers = np.moveaxis(m, 1, -1).reshape(-1, 40)
    empty = ~fibers.any(axis=1)
    # a fiber is empty when it was dropped (0.2) or when none of its 40
    # Bernoulli(0.05) draws came up (0.95^40 of the others)
    assert abs(empty.mean() - (0.2 + 0.8 * 0.95 ** 40)) < 0.03
    assert abs(m.mean() - 0.8 * 0.05) < 0.004


@pytest.mark.parametrize("name,dims,ranks,p,kind", [
    ("cube30_r3", (30, 30, 30), {(0, 1): 3, (0, 2): 3, (1, 2): 3}, 0.30, "max1"),
    ("msi256x256x31_r6", (256, 256, 31), {(0, 1): 6, (0, 2): 6, (1, 2): 6}, 0.10, "minmax01"),
    ("video144x176x3x100", (144, 176, 3, 100),
     {(0, 1): 8, (0, 3): 8, (1, 3): 8, (0, 2): 3, (1, 2): 3, (2, 3): 3}, 0.05, "minmax01"),
    ("traffic288x400x60x24_r5", (288, 400, 60, 24),
     {(k, l): 5 for k in range(4) for l in range(k + 1, 4)}, 0.05, "abs01"),
])
def test_workload_recipes_match_the_experiments(name, dims, ranks, p, kind):
    w = inp.WORKLOADS[name]
    assert w.dims == dims and w.p_observed == p and w.kind == kind and w.rho == 0.1
    for (k, l), r in ranks.items():
        assert w.R[k][l] == w.R[l][k] == r
    if name == "traffic288x400x60x24_r5":
        assert w.fiber == (1, 0.20)


@pytest.mark.parametrize("name", ["cube30_r3", "msi256x256x31_r6"])
def test_small_workloads_value_ranges_and_mask(name):
    w = inp.WORKLOADS[name]
    planted = oracle.reconstruct(w.dims, w.R, inp.gaussian_factors(w.dims, w.R, inp.planted_factor_seed(w)))
    xt, mask, G0 = inp.workload_inputs(w, planted)
    assert xt.shape == w.dims and xt.flags.c_contiguous
    if w.kind == "max1":
        assert np.max(np.abs(xt)) == 1.0
    else:
        assert xt.min() >= 0.0 and xt.max() <= 1.0
        # noise of the stated size on top of the min-max-scaled planted tensor
        lo, hi = planted.min(), planted.max()
        resid = (xt - (planted - lo) / (hi - lo))[(xt > 0) & (xt < 1)]
        assert abs(resid.std() - w.sigma) < 0.1 * w.sigma
    assert abs(mask.mean() - w.p_observed) < 0.01
    assert G0.size == inp.factor_size(w.dims, w.R) and G0.min() >= 0.0 and G0.max() < 1.0


def test_served_stream_requests_follow_the_stream_recipe():
    """512 requests, Poisson arrivals at 200/s, order 3 or 4 uniformly, modes
    uniform in [32, 128], per-edge ranks uniform in [2, 6], observed fraction
    uniform in [0.1, 0.5], 50 sweeps each."""
    from paper_2511_16358_gb300.serve_bench import draw_requests
    reqs = draw_requests(512, 200.0, 5000, 32, 128, 2, 6, 0.1, 0.5, 50)
    assert len(reqs) == 512
    t = np.array([r["t"] for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert (gaps > 0).all()
    assert abs(gaps.mean() - 1 / 200) < 0.15 / 200          # exponential: mean 1/rate
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.15       # and coefficient of variation 1
    orders = np.array([len(r["dims"]) for r in reqs])
    assert set(orders.tolist()) == {3, 4} and abs((orders == 4).mean() - 0.5) < 0.07
    dims = np.concatenate([r["dims"] for r in reqs])
    assert dims.min() == 32 and dims.max() == 128
    ranks = []
    for r in reqs:
        N = len(r["dims"])
        R = r["R"]
        assert (R == R.T).all()
        ranks += [int(R[k, l]) for k in range(N) for l in range(k + 1, N)]
    assert set(ranks) == {2, 3, 4, 5, 6}
    p = np.array([r["p"] for r in reqs])
    assert p.min() >= 0.1 and p.max() <= 0.5 and abs(p.mean() - 0.3) < 0.02
    assert all(r["sweeps"] == 50 for r in reqs)
