"""Failure handling on the device, and the default initial factors.

- Bounded waits: ifctn_wait_selftest runs the library's two device wait
  primitives -- the software grid barrier of the persistent sweep and the
  mbarrier phase wait of the TMA rings -- on conditions that nothing satisfies
  (a CTA that never arrives; bytes announced that no copy delivers), with a
  budget of a few thousand clock cycles.  Both give up, the kernel returns,
  and the call reports IFCTN_ETIMEOUT.  The CUDA context stays usable: the
  same library context then runs sweeps that match the oracle, and the flag
  is reported once (the next call returns OK).  Nothing here hangs or faults
  the GPU: every wait has a budget and the kernel returns.
- Default G^(0) (no initial factors given): seeded splitmix64 U(0,1)
  entries, rescaled by one common factor so that
  ||iFCTN(G^0)|| = ||P_Omega(O)|| / sqrt(|Omega|/P).  The library's start
  equals the same recipe computed with the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2511_16358_gb300 import binding as b
from tests._cases import make_case, rel_err, scaled_uniform_start

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [b.FP64, b.MIXED])
def test_bounded_waits_expire_report_timeout_and_context_stays_usable(precision):
    case = make_case((20, 18, 16), 3, 0.3, seed=401)
    dims, R = case["dims"], case["R"]
    dt = b.tensor_dtype(precision)
    c = b.Completion(dims, R, case["xt"].astype(dt), case["mask"], rho=0.1, max_sweeps=3, tol=0.0,
                     precision=precision, init_factors=case["G0"].copy())
    for _ in range(2):
        rc = b.wait_selftest(c.ctx, 5000)
        assert rc == b.ETIMEOUT, b.STATUS_NAMES[rc]
        assert "expired" in b.last_error()
    st = c.sweep(3)  # the flag was reported once and cleared: this call is clean
    assert st["sweeps_done"] == 3
    G, X = case["G0"].copy(), case["X0"].copy()
    oracle.complete(dims, R, 0.1, G, X, case["mask"], max_sweeps=3)
    tol = 1e-10 if precision == b.FP64 else 2e-3
    assert rel_err(c.factors(), G) < tol
    assert rel_err(c.x(), X) < tol
    assert b.load().ifctn_wait_selftest(c.ctx, 10) == b.EINVAL  # budget out of range
    c.close()


def test_default_initial_factors_follow_the_seeded_recipe():
    case = make_case((17, 15, 13, 6), 2, 0.25, seed=402)
    dims, R = case["dims"], case["R"]
    seed = 4321
    c = b.Completion(dims, R, case["xt"], case["mask"], rho=0.1, max_sweeps=1, tol=0.0, precision=b.FP64,
                     seed=seed)
    want = scaled_uniform_start(dims, R, case["X0"], case["mask"], seed)
    assert rel_err(c.factors(), want) < 1e-12
    np.testing.assert_array_equal(c.x(), case["X0"])
    c.close()
