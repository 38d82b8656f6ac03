"""Writes tucker20x4_rse.txt: the FP64 oracle's completion of the paper's
synthetic experiment (Sec. 5.1, Fig. 3) at every random-missing rate.

Truth: a 20x20x20x20 tensor of Tucker rank (5,5,5,5), U(0,1) core and
factors, scaled to [0, 1].  Completion: iFCTN with every R_{k,l} = 5, the
experiments' defaults rho = 0.1, t_max = 1000, eps = 1e-5 (Sec. 5), X^0 =
P_Omega(O), G^0 = seeded U(0,1) factors rescaled so that ||iFCTN(G^0)|| =
||P_Omega(O)|| / sqrt(p).  Every value comes from ``oracle/`` and the seeded
generators; nothing here touches the GPU library.

Run from the repository root:  python tests/golden/make_tucker20x4_rse.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2511_16358_gb300 import inputs as inp  # noqa: E402
from tests._cases import scaled_uniform_start  # noqa: E402

OUT = os.path.join(HERE, "tucker20x4_rse.txt")


def run(missing_rate, max_sweeps=None, nthreads=0):
    """Oracle completion of the Tucker workload at one missing rate; returns
    (sweeps done, per-sweep log, final X, X_true, mask)."""
    w = inp.WORKLOADS[f"tucker20x4_rm{int(round(100 * missing_rate)):02d}"]
    xt, mask, _ = inp.workload_inputs(w, None)
    X = oracle.init_x(xt, mask)
    G = scaled_uniform_start(w.dims, w.R, X, mask, 4000 + w.seed_base)
    log = oracle.complete(w.dims, w.R, w.rho, G, X, mask,
                          max_sweeps=w.sweeps if max_sweeps is None else max_sweeps,
                          tol=w.extra["tol"], xtrue=xt, nthreads=nthreads)
    return len(log), log, X, xt, mask


def main():
    rows = []
    for m in inp.TUCKER_MISSING_RATES:
        n, log, X, xt, mask = run(m)
        rse, rmse = oracle.metrics(xt, X, mask)
        rows.append((m, n, rse, rmse, log[-1]["rel_change"]))
        print(f"missing {m:.2f}: {n} sweeps, RSE {rse:.6e}, RMSE {rmse:.6e}", flush=True)
    with open(OUT, "w") as f:
        f.write("# The paper's synthetic experiment (Sec. 5.1, Fig. 3): 20^4 tensor of Tucker rank\n"
                "# (5,5,5,5), U(0,1) core and factors, scaled to [0,1]; iFCTN completion with every\n"
                "# R_{k,l} = 5, rho = 0.1, t_max = 1000, eps = 1e-5 (Sec. 5 defaults), FP64 oracle.\n"
                "# Written by tests/golden/make_tucker20x4_rse.py (oracle and seeded inputs only).\n"
                "# fields: missing_rate sweeps rse rmse final_rel_change\n")
        for m, n, rse, rmse, rc in rows:
            f.write(f"{m:.2f} {n} {rse:.17e} {rmse:.17e} {rc:.17e}\n")
    print(OUT)


if __name__ == "__main__":
    main()
