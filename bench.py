#!/usr/bin/env python
"""Benchmark of the iFCTN PAM sweep on one GB300 (or N replicas, one per GPU).

Workload (default): the multispectral-image shaped problem, 256 x 256 x 31
FP32 in [0,1], planted iFCTN with all ranks 6 plus N(0, 0.01^2) noise, 10%
uniformly observed, rho = 0.1, 100 sweeps per job, mixed precision.  One
"step" is one whole completion job (100 PAM sweeps) starting from the job's
initial state, which is restored from device-resident copies before the step;
L2 is flushed (a 256 MiB write) before every timed step.  The metric is PAM
sweeps per second over the whole job (all ranks).

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle instead (the reference arm of this benchmark).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PAM sweeps/s"
UNIT = "sweeps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="msi256x256x31_r6")
    ap.add_argument("--precision", default=None, choices=[None, "mixed", "fp64"])
    ap.add_argument("--quick", action="store_true", help="skip the FP64-path, time-to-RSE and e2e extras")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks sampling during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# workload inputs (planted with the library's own reconstruction)
# ---------------------------------------------------------------------------
def make_inputs(w, b, inp):
    dims, R = w.dims, w.R
    planted = None
    if w.planted:
        Gt = inp.gaussian_factors(dims, R, inp.planted_factor_seed(w))
        P = int(np.prod(dims))
        prob = b.make_problem(dims, R, rho=w.rho, max_sweeps=0, tol=0.0, precision=b.FP64)
        ctx = b.create(prob, np.zeros(P), np.zeros(P, dtype=np.uint8), Gt)
        planted = b.reconstruct(ctx, np.empty(dims, dtype=np.float64))
        b.destroy(ctx)
    xt, mask, _ = inp.workload_inputs(w, planted)
    return xt, mask


def time_steps(b, torch, ctx, stream, X0_dev, G0_dev, sweeps, steps, warmup, flush):
    times = []
    for it in range(warmup + steps):
        b.set_factors(ctx, G0_dev)
        b.set_x(ctx, X0_dev)
        with torch.cuda.stream(stream):
            flush.zero_()
            s = torch.cuda.Event(enable_timing=True)
            e = torch.cuda.Event(enable_timing=True)
            s.record(stream)
            b.sweep_async(ctx, sweeps)
            e.record(stream)
        stream.synchronize()
        if it >= warmup:
            times.append(s.elapsed_time(e) / 1000.0)
    st = b.sweep(ctx, 0)  # surfaces any device-side failure
    return times, st


def stage_times(b, torch, ctx, stream, N, reps=20):
    """Average device time per launch of each stage (CUDA events on the
    context's stream around back-to-back launches)."""
    from paper_2511_16358_gb300.stage_timer import time_stage
    out = {}
    for stage, name in ((0, "contract"), (4, "finish"), (1, "gram"), (2, "solve"), (3, "xupdate")):
        modes = range(N) if stage != 3 else [0]
        for k in modes:
            out[f"{name}{k}" if stage != 3 else name] = time_stage(torch, b, ctx, stream, stage, k, reps)
    return out


def rse_curve(b, ctx, xt, sweeps):
    b.set_truth(ctx, xt, log=True)
    b.sweep(ctx, sweeps)
    log = b.get_log(ctx)
    return [r["rse"] for r in log[-sweeps:]]


def aggregate_ranks(torch, dist, seconds, world, units_per_rank, device):
    """Whole-job throughput of N replicas: every rank timed the same amount of
    work; the job took as long as the slowest rank (MAX over ranks), and the
    units of all ranks count.  Returns (max seconds, units per second)."""
    if dist is not None and world > 1:
        t = torch.tensor([seconds], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        seconds = float(t.item())
    return seconds, world * units_per_rank / seconds


def source_digest() -> str:
    """Digest of the CUDA sources (as in the build stamp, without the flags)."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2511_16358_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def committed_traffic(kernel: str, workload: str):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of
    ``kernel`` on ``workload`` from the committed ncu summary, or None when the
    summary was taken on other kernel sources than the ones built here."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    dig = source_digest()
    for ln in lines:
        f = dict(kv.split("=", 1) for kv in ln.split() if "=" in kv)
        if f.get("kernel") == kernel and f.get("workload") == workload and f.get("digest") == dig:
            return float(f["bytes_per_launch"])
    return None


def cpu_baseline(w, budget_s=15.0):
    import oracle
    from paper_2511_16358_gb300 import inputs as inp
    dims, R = w.dims, w.R
    planted = (oracle.reconstruct(dims, R, inp.gaussian_factors(dims, R, inp.planted_factor_seed(w)))
               if w.planted else None)
    xt, mask, G0 = inp.workload_inputs(w, planted)
    X = oracle.init_x(xt, mask)
    rec = oracle.reconstruct(dims, R, G0)
    N = len(dims)
    G = G0 * (np.linalg.norm(X) / np.sqrt(w.p_observed) / np.linalg.norm(rec)) ** (1.0 / (N * (N - 1)))
    cores = os.cpu_count() or 1
    n, t0 = 0, time.perf_counter()
    while True:
        oracle.sweep(dims, R, w.rho, G, X, mask, nthreads=cores)
        n += 1
        el = time.perf_counter() - t0
        if el > budget_s or n >= 2000:
            break
    return {"value": n / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} FP64 oracle sweeps of {w.name} on {cores} host threads ({el:.1f} s)"}


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2511_16358_gb300 import inputs as inp
    dims, R = w.dims, w.R
    planted = (oracle.reconstruct(dims, R, inp.gaussian_factors(dims, R, inp.planted_factor_seed(w)))
               if w.planted else None)
    xt, mask, G0 = inp.workload_inputs(w, planted)
    X = oracle.init_x(xt, mask)
    rec = oracle.reconstruct(dims, R, G0)
    N = len(dims)
    G = G0 * (np.linalg.norm(X) / np.sqrt(w.p_observed) / np.linalg.norm(rec)) ** (1.0 / (N * (N - 1)))
    cores = os.cpu_count() or 1
    per = []
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.sweep(dims, R, w.rho, G, X, mask, nthreads=cores)
        if it >= args.warmup:
            per.append(time.perf_counter() - t0)
    tot = sum(per)
    v = len(per) / tot
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / len(per),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w.name, "dims": list(dims), "sweeps_per_step": 1,
                                             "implementation": "FP64 CPU oracle (C, OpenMP)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"1 oracle sweep of {w.name} per step, {cores} host threads"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    from paper_2511_16358_gb300 import inputs as inp
    w = inp.WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, w)
        return
    import torch
    # the persistent kernel timestamps the phases of one sweep of every launch:
    # a sweep from the middle of the step (steady state), unless set otherwise
    os.environ.setdefault("IFCTN_STAMP_SWEEP", str(max(0, w.sweeps // 2)))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__
    __graft_entry__.build()
    from paper_2511_16358_gb300 import binding as b

    prec = b.MIXED if (args.precision or w.precision) == "mixed" else b.FP64
    dt = b.tensor_dtype(prec)
    sweeps = w.sweeps
    xt, mask = make_inputs(w, b, inp)
    P = xt.size
    dims = w.dims
    N = len(dims)
    stream = torch.cuda.Stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MiB > L2

    def new_ctx(precision, n):
        return b.create(b.make_problem(dims, w.R, rho=w.rho, max_sweeps=n, tol=0.0, precision=precision,
                                       seed=4000 + w.seed_base),
                        xt.astype(b.tensor_dtype(precision)), mask, None, stream.cuda_stream)

    ctx = new_ctx(prec, sweeps)
    G0 = torch.empty(inp.factor_size(dims, w.R), dtype=torch.float64, device="cuda")
    b.get_factors(ctx, G0)
    X0 = torch.empty(dims, dtype=torch.float32 if dt == np.float32 else torch.float64, device="cuda")
    b.get_x(ctx, X0)
    kps = b.kernels_per_sweep(ctx)

    clocks = Clocks(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    lc0 = b.launch_count(ctx)
    times, st_last = time_steps(b, torch, ctx, stream, X0, G0, sweeps, args.steps, args.warmup, flush)
    ck = clocks.stop()
    launches_timed = (b.launch_count(ctx) - lc0) * args.steps // (args.steps + args.warmup)
    ph = b.phase_times(ctx)
    names = []
    for k in range(len(w.dims)):
        names += [f"m{k}_contract", f"m{k}_bar1", f"m{k}_reduce", f"m{k}_bar2", f"m{k}_solve", f"m{k}_bar3"]
    names = names[: 6 * len(w.dims)]
    phases = {}
    prev = 0.0
    for nm, t in zip(names, ph[: 6 * len(w.dims)]):
        phases[nm] = t - prev
        prev = t
    if len(ph) >= 26:
        phases["xupdate"] = ph[24] - prev
        phases["xupdate_bar"] = ph[25] - ph[24]
    for k in range(len(w.dims)):
        if len(ph) >= 28 + 2 * k:
            phases[f"m{k}_contract_cta_max_end"] = ph[26 + 2 * k]
            phases[f"m{k}_contract_cta_mean_end"] = ph[27 + 2 * k]
    sub = ph[26 + 2 * N: 26 + 2 * N + 12]
    if len(sub) == 12:
        names_sub = ["start", "staged", "column_loaded", "omega", "H_b_sums", "reduced", "ldlt_solve", "refined",
                     "checked", "stored", "stages_done", "W_refreshed"]
        mode = int(os.environ.get("IFCTN_STAMP_MODE", len(w.dims) - 1))
        phases["solve_first_column_s"] = {nm: (t - sub[0]) for nm, t in zip(names_sub, sub)}
        phases["solve_first_column_s"]["mode"] = mode
    red = ph[26 + 2 * N + 12: 26 + 2 * N + 16]
    if len(red) == 4 and red[0] == red[0]:
        phases["reduce_substeps_s"] = {"K_done": red[1] - red[0], "coef_done": red[2] - red[0],
                                       "M_done": red[3] - red[0]}
    torch.cuda.synchronize()
    tot, value = aggregate_ranks(torch, dist, sum(times), world, args.steps * sweeps, "cuda")

    extras = {}
    # per-stage device times (separate context: stages mutate the state)
    pctx = new_ctx(prec, sweeps)
    stt = stage_times(b, torch, pctx, stream, N)
    b.destroy(pctx)
    sz = np.dtype(dt).itemsize
    per_sweep = {}
    for key, v in stt.items():
        base = key.rstrip("0123456789")
        per_sweep[base] = per_sweep.get(base, 0.0) + v
    dominant = max(per_sweep, key=per_sweep.get)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    src = "measured" if "hbm_gbs" in peaks else "fallback"
    mask_bytes = (P + 7) // 8
    sweep_bytes = (N + 2) * P * sz + mask_bytes  # N contraction reads, X read + write, mask
    persistent = launches_timed == args.steps  # one launch per step
    if persistent:
        # one cooperative launch runs the whole step (all sweeps); its device
        # time is the CUDA-event time of the step on the context's stream
        kname = "k_sweep_persistent (all phases of all sweeps, one cooperative launch)"
        alg = sweeps * sweep_bytes
        t_launch = tot / args.steps
    else:
        kname = "k_contract_roww/k_contract_colw (mode-k streaming contraction, warp-pipelined)"
        alg = P * sz  # one read of X per contraction launch
        t_launch = sum(v for kk, v in stt.items() if kk.startswith("contract")) / N
    achieved = alg / t_launch / 1e9
    roofline = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "peak_source": src,
                "algorithmic_bytes_per_launch": alg, "seconds_per_launch": t_launch,
                "traffic": committed_traffic(kname.split()[0], w.name),
                "stage_seconds_per_launch": stt,
                "stage_share_per_sweep": {k: v / sum(per_sweep.values()) for k, v in per_sweep.items()},
                "dominant_stage": dominant}
    if persistent:
        roofline["note"] = ("tensor resident in L2 (%.1f MB): the sweep is bound by the latency of its "
                            "dependent phases, not by HBM" % (P * sz / 1e6))

    if not args.quick and rank == 0:
        # plain FP64 GPU path on the same job
        if prec == b.MIXED:
            c64 = new_ctx(b.FP64, sweeps)
            G064 = torch.empty_like(G0)
            b.get_factors(c64, G064)
            X064 = torch.empty(dims, dtype=torch.float64, device="cuda")
            b.get_x(c64, X064)
            t64, _ = time_steps(b, torch, c64, stream, X064, G064, sweeps, max(1, min(args.steps, 3)), 1, flush)
            v64 = sweeps * len(t64) / sum(t64)
            extras["fp64_path"] = {"value": v64, "unit": UNIT, "speedup_mixed_over_fp64": value / world / v64}
            # time-to-RSE: RSE* = FP64 RSE after the job's sweeps x (1 + 1e-3)
            b.set_factors(c64, G064)
            b.set_x(c64, X064)
            r64 = rse_curve(b, c64, xt.astype(np.float64), sweeps)
            b.set_factors(ctx, G0)
            b.set_x(ctx, X0)
            r32 = rse_curve(b, ctx, xt.astype(np.float32), sweeps)
            target = r64[-1] * (1 + 1e-3)
            s32 = next((i + 1 for i, r in enumerate(r32) if r <= target), None)
            s64 = next((i + 1 for i, r in enumerate(r64) if r <= target), None)
            extras["time_to_rse"] = {
                "rse_target": target, "rse_fp64_final": r64[-1], "rse_mixed_final": r32[-1],
                "sweeps_mixed": s32, "sweeps_fp64": s64,
                "seconds_mixed": (s32 / (value / world)) if s32 else None,
                "seconds_fp64": (s64 / v64) if s64 else None}
            b.destroy(c64)
        # end to end through the public API with host buffers
        import torch as _t
        obs_h = _t.from_numpy(xt.astype(dt)).pin_memory()
        mask_h = _t.from_numpy(mask.astype(np.uint8)).pin_memory()
        out_h = _t.empty(dims, dtype=obs_h.dtype).pin_memory()
        e2e = []
        for it in range(2 + args.steps):
            t0 = time.perf_counter()
            c = b.create(b.make_problem(dims, w.R, rho=w.rho, max_sweeps=sweeps, tol=0.0, precision=prec,
                                        seed=4000 + w.seed_base), obs_h, mask_h, None, None)
            b.complete(c, out_h)
            b.destroy(c)
            if it >= 2:
                e2e.append(time.perf_counter() - t0)
        extras["e2e"] = {"value": sweeps * len(e2e) / sum(e2e), "unit": UNIT,
                         "h2d_bytes_per_step": int(P * (sz + 1)), "d2h_bytes_per_step": int(P * sz)}
        extras["cpu_baseline"] = cpu_baseline(w)
    b.destroy(ctx)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1000 * tot / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == b.MIXED else "f64",
                "data": "synthetic",
                "config": {"workload": w.name, "dims": list(dims), "ranks": int(w.R[0][1]),
                           "observed": w.p_observed, "sweeps_per_step": sweeps,
                           "precision": "mixed (FP32 tensor/contractions, FP64 solves)" if prec == b.MIXED else "fp64",
                           "l2": "flushed (256 MiB write) before every timed step",
                           "parallelism": f"replicas x{world}"},
                "gpu_launches": launches_timed,
                "persistent_phases_s": dict(phases, sweep=int(os.environ["IFCTN_STAMP_SWEEP"])),
                "clocks": ck, "roofline": roofline}
        line.update(extras)
        line.setdefault("e2e", None)
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
