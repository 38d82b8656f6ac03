"""GPU path on the paper's synthetic experiment (Sec. 5.1, Fig. 3), through the C ABI.

Truth: 20^4 tensor of Tucker rank (5,5,5,5), U(0,1) core and factors, scaled
to [0,1]; iFCTN completion with every R_{k,l} = 5 at 90 % random missing,
rho = 0.1.  FP64 path: factors and tensor within 1e-10 relative of the oracle
after a fixed number of sweeps (both execution paths), and the convergence run
at the experiments' defaults (t_max = 1000, eps = 1e-5) stops at the same
sweep as the stored oracle run with the same RSE.  Mixed path: RSE within
1e-3 relative of the oracle's.
"""
import os
import sys

import numpy as np
import pytest

import oracle
from paper_2511_16358_gb300 import binding as b
from paper_2511_16358_gb300 import inputs as inp
from tests._cases import path, rel_err, scaled_uniform_start

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_tucker20x4_rse as mk  # noqa: E402

pytestmark = pytest.mark.gpu

W = inp.WORKLOADS["tucker20x4_rm90"]


def _case():
    xt, mask, _ = inp.workload_inputs(W, None)
    X0 = oracle.init_x(xt, mask)
    G0 = scaled_uniform_start(W.dims, W.R, X0, mask, 4000 + W.seed_base)
    return xt, mask, X0, G0


def _golden_row(missing):
    with open(os.path.join(HERE, "golden", "tucker20x4_rse.txt")) as f:
        for ln in f:
            if ln.startswith("#") or not ln.strip():
                continue
            m, n, rse, rmse, rc = ln.split()
            if abs(float(m) - missing) < 1e-9:
                return int(n), float(rse), float(rmse)
    raise KeyError(missing)


@pytest.mark.parametrize("which", ["persistent", "graph"])
def test_fixed_sweeps_fp64_matches_oracle(which):
    xt, mask, X0, G0 = _case()
    n = 30
    with path(which):
        c = b.Completion(W.dims, W.R, xt, mask, rho=W.rho, max_sweeps=n, tol=0.0,
                         precision=b.FP64, init_factors=G0.copy())
    c.sweep(n)
    G, X = G0.copy(), X0.copy()
    oracle.complete(W.dims, W.R, W.rho, G, X, mask, max_sweeps=n)
    assert rel_err(c.factors(), G) < 1e-10
    assert rel_err(c.x(), X) < 1e-10
    c.close()


def test_paper_default_convergence_matches_stored_oracle_run():
    xt, mask, X0, G0 = _case()
    c = b.Completion(W.dims, W.R, xt, mask, rho=W.rho, max_sweeps=W.sweeps, tol=W.extra["tol"],
                     precision=b.FP64, init_factors=G0.copy())
    st = c.complete()
    n, rse, rmse = _golden_row(0.9)
    assert st["sweeps_done"] == n and st["converged"] == 1
    rse_g, rmse_g = oracle.metrics(xt, c.x(), mask)
    assert abs(rse_g - rse) <= 1e-9 * rse
    assert abs(rmse_g - rmse) <= 1e-9 * rmse
    c.close()


def test_mixed_rse_within_bound_of_oracle():
    n_conv, _, _ = _golden_row(0.9)
    xt, mask, X0, G0 = _case()
    c = b.Completion(W.dims, W.R, xt.astype(np.float32), mask, rho=W.rho, max_sweeps=n_conv,
                     tol=0.0, precision=b.MIXED, init_factors=G0.copy())
    c.sweep(n_conv)
    n, log, X, _, _ = mk.run(0.9)
    rse_o, _ = oracle.metrics(xt, X, mask)
    rse_g, _ = oracle.metrics(xt, c.x().astype(np.float64), mask)
    assert abs(rse_g - rse_o) <= 1e-3 * rse_o, (rse_g, rse_o)
    c.close()
