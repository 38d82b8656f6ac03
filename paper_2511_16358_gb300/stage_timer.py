"""Per-stage device times of one PAM sweep for a given problem shape.

    python -m paper_2511_16358_gb300.stage_timer --dims 288,400,60,24 --rank 5 --sweeps 2

Builds a problem with seeded uniform data and a 5 % uniform mask, runs the
requested sweeps through the public API, then times every stage kernel of the
sweep (contraction, Gram, solve per mode; X update) with CUDA events on the
context's stream and prints one JSON line.  Stage launches mutate the state,
so the stage times come after the sweeps whose statistics are reported.
Used to profile single kernels under ncu on shapes smaller than a workload.
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def time_stage(torch, b, ctx, stream, stage, k, reps):
    """Device seconds per launch of one stage: CUDA events on the context's
    stream around ``reps`` back-to-back launches (after two warm-up ones)."""
    for _ in range(2):
        b.launch_stage(ctx, stage, k)
    stream.synchronize()
    with torch.cuda.stream(stream):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            b.launch_stage(ctx, stage, k)
        e1.record(stream)
    stream.synchronize()
    return e0.elapsed_time(e1) / 1000.0 / reps


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", default="288,400,60,8")
    ap.add_argument("--rank", type=int, default=5)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--sweeps", type=int, default=2)
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--observed", type=float, default=0.05)
    ap.add_argument("--stages", default="contract,finish,gram,solve,xupdate")
    args = ap.parse_args(argv)

    import torch

    from . import binding as b
    from . import inputs as inp

    dims = tuple(int(x) for x in args.dims.split(","))
    R = inp.rank_matrix(len(dims), args.rank)
    prec = b.MIXED if args.precision == "mixed" else b.FP64
    dt = b.tensor_dtype(prec)
    P = int(np.prod(dims))
    xt = inp.uniform(7, P).astype(dt).reshape(dims)
    mask = (inp.uniform(8, P) < args.observed).astype(np.uint8).reshape(dims)
    stream = torch.cuda.Stream()
    ctx = b.create(b.make_problem(dims, R, rho=0.1, max_sweeps=max(args.sweeps, 1), tol=0.0, precision=prec,
                                  seed=9), xt, mask, None, stream.cuda_stream)
    st = b.sweep(ctx, args.sweeps)
    b.sweep(ctx, 0)  # surfaces any device-side failure of the sweeps
    out = {"dims": list(dims), "rank": args.rank, "precision": args.precision, "sweeps": st,
           "kernels_per_sweep": b.kernels_per_sweep(ctx), "stage_us": {}}
    want = set(args.stages.split(","))
    for stage, name in ((0, "contract"), (4, "finish"), (1, "gram"), (2, "solve"), (3, "xupdate")):
        if name not in want:
            continue
        for k in (range(len(dims)) if stage != 3 else [0]):
            key = f"{name}{k}" if stage != 3 else name
            out["stage_us"][key] = time_stage(torch, b, ctx, stream, stage, k, args.reps) * 1e6
    # Repeating one stage out of order moves the state away from a sweep's
    # (e.g. solves against a stale Gram matrix), so a status raised now says
    # nothing about the sweep and is only reported.
    try:
        b.sweep(ctx, 0)
        out["after_stage_timing"] = "ok"
    except b.IfctnError as e:
        out["after_stage_timing"] = str(e)
    b.destroy(ctx)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
