"""Writes workload_rse.txt: the FP64 oracle's RSE along a whole benchmark job.

For each experiment-shaped workload (multispectral 256x256x31, colour video
144x176x3x100, traffic 288x400x60x24) the oracle runs the workload's fixed
number of PAM sweeps (Algorithm 1 with tol = 0) from the job's start:
X^0 = P_Omega(O) and G^0 = the seeded U(0,1) factors (seed 4000 + the
workload's seed base) rescaled by one common factor so that
||iFCTN(G^0)|| = ||P_Omega(O)|| / sqrt(p).  It records the RSE
||X_true - X^s|| / ||X_true|| (Sec. 5) after selected sweeps s and the RMSE
over the missing entries at the end.  The benchmark states the error of the
GPU paths' RSE against these values.  Every value comes from ``oracle/`` and
the seeded generators; nothing here touches the GPU library.

Run from the repository root:
    python tests/golden/make_workload_rse.py [workload ...]
The traffic workload takes about half an hour on 8 host threads (200 oracle
sweeps of a 166M-entry tensor); lines of workloads not given are kept.
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2511_16358_gb300 import inputs as inp  # noqa: E402
from tests._cases import scaled_uniform_start  # noqa: E402

OUT = os.path.join(HERE, "workload_rse.txt")
NAMES = ("msi256x256x31_r6", "video144x176x3x100", "traffic288x400x60x24_r5")


def checkpoints(n):
    return sorted({1, 2, 5, 10, 20, 40, 50, 72, 100, 150, 200, n} & set(range(1, n + 1)))


def run(name, nthreads=0):
    w = inp.WORKLOADS[name]
    planted = oracle.reconstruct(w.dims, w.R, inp.gaussian_factors(w.dims, w.R, inp.planted_factor_seed(w)))
    xt, mask, _ = inp.workload_inputs(w, planted)
    del planted
    X = oracle.init_x(xt, mask)
    G = scaled_uniform_start(w.dims, w.R, X, mask, 4000 + w.seed_base)
    marks = checkpoints(w.sweeps)
    out, done, t0 = [], 0, time.time()
    for s in marks:
        oracle.complete(w.dims, w.R, w.rho, G, X, mask, max_sweeps=s - done, tol=0.0, nthreads=nthreads)
        done = s
        rse, rmse = oracle.metrics(xt, X, mask)
        out.append((s, rse, rmse))
        print(f"{name}: sweep {s}: RSE {rse:.10e} ({time.time() - t0:.0f} s)", flush=True)
    return out


def read(path=OUT):
    """{workload: {sweep: (rse, rmse)}} from the golden file."""
    rows = {}
    if not os.path.exists(path):
        return rows
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, s, rse, rmse = line.split()
        rows.setdefault(name, {})[int(s)] = (float(rse), float(rmse))
    return rows


def main(names):
    rows = read()
    for name in names:
        rows[name] = {s: (rse, rmse) for s, rse, rmse in run(name)}
    with open(OUT, "w") as f:
        f.write("# FP64 oracle RSE = ||X_true - X^s|| / ||X_true|| (Sec. 5) after sweep s of each\n"
                "# benchmark workload's fixed-length PAM job (Algorithm 1, tol = 0), from X^0 = P_Omega(O)\n"
                "# and the seeded, rescaled U(0,1) start G^0 (seed 4000 + seed base); RMSE over the missing\n"
                "# entries.  Written by tests/golden/make_workload_rse.py (oracle and seeded inputs only).\n"
                "# fields: workload sweep rse rmse\n")
        for name in NAMES:
            for s, (rse, rmse) in sorted(rows.get(name, {}).items()):
                f.write(f"{name} {s} {rse:.17e} {rmse:.17e}\n")
    print(OUT)


if __name__ == "__main__":
    main(sys.argv[1:] or list(NAMES))
