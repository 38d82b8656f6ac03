"""The autotuner's selection rule, on fake timings (no GPU): the planner's
default (first candidate) is kept unless the fastest candidate beats it by
2 % or more; otherwise the fastest wins, the earliest of equal ones."""
import pytest


@pytest.fixture(scope="module")
def b():
    from paper_2511_16358_gb300 import _build, binding
    _build.build()
    binding.load()
    return binding


@pytest.mark.parametrize("secs,want", [
    ([1.0], 0),
    ([1.0, 0.99, 0.995], 0),        # 1 % faster: noise, the default stays
    ([1.0, 0.97, 0.98], 1),         # 3 % faster: taken
    ([1.0, 0.90, 0.80, 0.80], 2),   # fastest; the earlier of two equal ones
    ([0.5, 1.0, 2.0], 0),           # the default is the fastest
    ([1.0, 0.98], 1),               # exactly 2 %
])
def test_tune_choose_rule(b, secs, want):
    assert b.tune_choose(secs) == want


def test_tune_choose_rejects_empty(b):
    assert b.tune_choose([]) == -1
    assert b.load().ifctn_tune_choose(3, None) == -1
