"""The autotuner on the GPU: it times the contraction's candidate launch
shapes once per shape, records its choices in the cache file, answers later
contexts of the same shape from the cache without timing anything, and a
tuned context still matches the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2511_16358_gb300 import binding as b
from tests._cases import make_case, path, rel_err

pytestmark = pytest.mark.gpu


def _ctx(case, precision, n):
    dt = b.tensor_dtype(precision)
    with path("graph"):
        return b.Completion(case["dims"], case["R"], case["xt"].astype(dt), case["mask"], rho=0.1, max_sweeps=n,
                            tol=0.0, precision=precision, init_factors=case["G0"].copy())


def test_tuner_times_once_caches_and_keeps_parity(tmp_path, monkeypatch):
    cache = tmp_path / "tune.txt"
    case = make_case((12, 14, 50, 12), 3, 0.3, seed=471, kind="max1", sigma=0.02)
    c = _ctx(case, b.FP64, 2)
    timed = b.tune(c.ctx, cache)
    assert timed >= 2  # at least the default and one alternative per tuned mode
    lines = [ln for ln in cache.read_text().splitlines() if ln.startswith("ifctn-tune-v1 ")]
    assert len(lines) == 4  # every mode of this shape runs the warp-pipelined kernels
    assert all(" f64 " in ln and "N4,12,14,50,12" in ln for ln in lines)
    c.sweep(2)
    G, X = case["G0"].copy(), case["X0"].copy()
    oracle.complete(case["dims"], case["R"], 0.1, G, X, case["mask"], max_sweeps=2)
    assert rel_err(c.factors(), G) < 1e-10
    assert rel_err(c.x(), X) < 1e-10
    c.close()
    # a second context of the shape is tuned at creation from the cache alone
    monkeypatch.setenv("IFCTN_TUNE_CACHE", str(cache))
    c2 = _ctx(case, b.FP64, 2)
    assert b.tune(c2.ctx, cache) == 0
    assert len(cache.read_text().splitlines()) == 4
    c2.sweep(2)
    assert rel_err(c2.factors(), G) < 1e-10
    c2.close()


def test_tuner_mixed_precision_and_ignores_malformed_lines(tmp_path):
    cache = tmp_path / "tune.txt"
    cache.write_text("ifctn-tune-v1 garbage\nnot a line\n")
    case = make_case((10, 9, 40, 16), 4, 0.3, seed=472, kind="max1", sigma=0.02)
    c = _ctx(case, b.MIXED, 3)
    assert b.tune(c.ctx, cache) >= 2
    assert b.tune(c.ctx, cache) == 0  # answered by the lines just written
    c.sweep(3)
    G, X = case["G0"].copy(), case["X0"].copy()
    oracle.complete(case["dims"], case["R"], 0.1, G, X, case["mask"], max_sweeps=3)
    assert rel_err(c.x().astype(np.float64), X) < 2e-3
    c.close()


def test_execution_path_choice_is_timed_once_and_cached(tmp_path, monkeypatch):
    """A tensor small enough for the one-launch persistent path: creation with
    a tuning cache times both execution paths, keeps the faster, records the
    choice; a later creation of the shape reads it; both match the oracle."""
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("IFCTN_TUNE_CACHE", str(cache))
    monkeypatch.delenv("IFCTN_PATH", raising=False)
    case = make_case((16, 15, 6, 20), {(0, 1): 3, (0, 2): 2, (0, 3): 3, (1, 2): 2, (1, 3): 3, (2, 3): 2}, 0.3,
                     seed=473, kind="max1", sigma=0.02)
    G, X = case["G0"].copy(), case["X0"].copy()
    oracle.complete(case["dims"], case["R"], 0.1, G, X, case["mask"], max_sweeps=3)
    for attempt in range(2):
        c = b.Completion(case["dims"], case["R"], case["xt"], case["mask"], rho=0.1, max_sweeps=3, tol=0.0,
                         precision=b.FP64, init_factors=case["G0"].copy())
        paths = [ln for ln in cache.read_text().splitlines() if " path " in ln]
        assert len(paths) == 1 and (" path=graph " in paths[0] or " path=persistent " in paths[0])
        st = c.sweep(3)
        assert st["sweeps_done"] == 3  # timing sweeps left no trace in the state or the log
        assert rel_err(c.factors(), G) < 1e-10
        assert rel_err(c.x(), X) < 1e-10
        c.close()
