"""Serving through the C ABI: continuous batching of completion jobs.

- A job's result is the same alone and in a mix of jobs of other orders,
  sizes, ranks and precisions that are resident at the same time (bitwise:
  every job runs the kernel code it would run alone, in the same order; jobs
  whose tensors stay in L2 share cooperative launches, each on its own slice
  of the grid, and the persistent kernel's results do not depend on the grid).
- Its result equals the oracle's (FP64 path within 1e-10).
- Admission follows the device-memory budget: with room for one job at a
  time, jobs run one after another and all complete.
- poll: ENOTREADY without waiting, ETIMEOUT with a short wait, ENOTFOUND for a
  released ticket; a job larger than the budget is refused at submit.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2511_16358_gb300 import binding as b
from tests._cases import make_case, rel_err

pytestmark = pytest.mark.gpu

GB = 1 << 30


def _problem(case, precision, sweeps, seed=0):
    return b.make_problem(case["dims"], case["R"], rho=0.1, max_sweeps=sweeps, tol=0.0, precision=precision,
                          seed=seed)


def _submit(srv, case, precision, sweeps, with_init=True):
    dt = b.tensor_dtype(precision)
    return b.submit(srv, _problem(case, precision, sweeps), case["xt"].astype(dt), case["mask"],
                    case["G0"].copy() if with_init else None)


def _collect(srv, ticket, case, precision):
    out = np.empty(case["dims"], dtype=b.tensor_dtype(precision))
    rc, st = b.poll(srv, ticket, out, timeout_us=-1)
    assert rc == b.OK
    return out, st


JOBS = [
    (((12, 11, 10), 3, 0.3, 201), b.FP64, 6),
    (((9, 8, 7, 6), {(0, 1): 2, (0, 2): 3, (0, 3): 2, (1, 2): 4, (1, 3): 2, (2, 3): 3}, 0.4, 202), b.MIXED, 8),
    (((40, 36, 31), 4, 0.2, 203), b.MIXED, 10),
    (((7, 6, 5, 8), 2, 0.5, 204), b.FP64, 5),
    (((20, 18, 16), 5, 0.1, 205), b.MIXED, 12),
]


def test_result_same_alone_and_in_the_mix_and_matches_oracle():
    cases = [make_case(d, e, p, seed=s) for (d, e, p, s), _, _ in JOBS]
    # alone: one job resident at a time
    srv = b.server_create(64 * GB, 1)
    alone = []
    for case, (_, prec, n) in zip(cases, JOBS):
        t = _submit(srv, case, prec, n)
        alone.append(_collect(srv, t, case, prec)[0])
    b.server_destroy(srv)
    # in the mix: all submitted at once, up to 4 resident together
    srv = b.server_create(64 * GB, 4)
    tickets = [_submit(srv, case, prec, n) for case, (_, prec, n) in zip(cases, JOBS)]
    mixed = [_collect(srv, t, case, prec)[0] for t, case, (_, prec, _n) in zip(tickets, cases, JOBS)]
    info = b.server_info_get(srv)
    b.server_destroy(srv)
    assert info["completed"] == len(JOBS)
    assert info["peak_resident"] >= 2
    # these tensors stay in L2: their sweeps ran in shared persistent launches,
    # several jobs a launch
    assert info["batch_launches"] > 0 and info["batched_jobs"] > info["batch_launches"]
    for a, m in zip(alone, mixed):
        np.testing.assert_array_equal(a, m)
    # FP64 jobs against the oracle
    for case, (_, prec, n), x in zip(cases, JOBS, mixed):
        if prec != b.FP64:
            continue
        G, X = case["G0"].copy(), case["X0"].copy()
        oracle.complete(case["dims"], case["R"], 0.1, G, X, case["mask"], max_sweeps=n)
        assert rel_err(x, X) < 1e-10


def test_admission_by_budget_runs_jobs_one_at_a_time():
    case = make_case((24, 22, 20), 3, 0.3, seed=211)
    # each job needs about 9 bytes per entry plus 8 MiB of slack: room for one
    srv = b.server_create(12 << 20, 8)
    tickets = [_submit(srv, case, b.MIXED, 4) for _ in range(4)]
    outs = [_collect(srv, t, case, b.MIXED)[0] for t in tickets]
    info = b.server_info_get(srv)
    b.server_destroy(srv)
    assert info["completed"] == 4
    assert info["peak_resident"] == 1
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])


def test_poll_not_ready_timeout_and_released_ticket():
    case = make_case((40, 36, 31), 6, 0.2, seed=221)
    srv = b.server_create(64 * GB, 1)
    t0 = _submit(srv, case, b.FP64, 300)  # long enough to be running when polled
    rc, _ = b.poll(srv, t0, None, timeout_us=0)
    assert rc in (b.ENOTREADY, b.OK)
    if rc == b.ENOTREADY:
        rc2, _ = b.poll(srv, t0, None, timeout_us=100)
        assert rc2 in (b.ETIMEOUT, b.OK)
        if rc2 == b.ETIMEOUT:
            rc3, st = b.poll(srv, t0, None, timeout_us=-1)
            assert rc3 == b.OK and st["sweeps_done"] == 300
    with pytest.raises(b.IfctnError):
        b.poll(srv, t0, None, timeout_us=0)  # ticket released
    assert b.server_latency(srv, t0) > 0
    b.server_destroy(srv)


def test_job_larger_than_budget_is_refused():
    case = make_case((30, 30, 30), 3, 0.3, seed=231)
    srv = b.server_create(1 << 20, 2)
    with pytest.raises(b.IfctnError):
        _submit(srv, case, b.MIXED, 2)
    b.server_destroy(srv)


def test_served_default_initial_factors_are_seeded():
    """Jobs without initial factors start from the seeded default: the same
    seed gives the same result, served or not."""
    case = make_case((16, 15, 14), 3, 0.3, seed=241)
    srv = b.server_create(64 * GB, 2)
    t1 = _submit(srv, case, b.MIXED, 5, with_init=False)
    x1, _ = _collect(srv, t1, case, b.MIXED)
    b.server_destroy(srv)
    c = b.Completion(case["dims"], case["R"], case["xt"].astype(np.float32), case["mask"], rho=0.1, max_sweeps=5,
                     tol=0.0, precision=b.MIXED)
    c.sweep(5)
    np.testing.assert_array_equal(c.x(), x1)
    c.close()
    time.sleep(0)
