"""The slab-sharded sweep through the library, two processes on one GPU.

The tensor is split along its first mode into two slabs; each process (a
gloo rank) holds one slab in its own context on cuda:0 and runs
ifctn_sweep_exchange, which combines the partial M_k and K_k of the modes
k >= 2 (1-based) and the stop-test sums with the ordered allreduce over gloo
between kernel launches (no kernel waits on the other process).  The merged
factors and the concatenated slabs of X equal the FP64 oracle's sweeps of the
whole problem within 1e-10, the factors of the modes the slabs share are
bitwise equal on both processes, and the stop-test values match the oracle's.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_2511_16358_gb300 import sharding as sh
from tests._cases import make_case, rel_err

pytestmark = pytest.mark.gpu

SWEEPS = 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, case, precision, exec_path, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), IFCTN_PATH=exec_path)
    import torch
    import torch.distributed as dist

    from paper_2511_16358_gb300 import binding as b
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dims, R = case["dims"], case["R"]
    lo, hi = sh.slab_bounds(dims[0], world, rank)
    sdims = (hi - lo,) + tuple(dims[1:])
    dt = b.tensor_dtype(precision)
    c = b.Completion(sdims, R, np.ascontiguousarray(case["xt"][lo:hi]).astype(dt),
                     np.ascontiguousarray(case["mask"][lo:hi]), rho=0.1, max_sweeps=SWEEPS, tol=0.0,
                     precision=precision, init_factors=sh.slab_factors(case["G0"], dims, R, lo, hi))
    st = b.sweep_exchange(c.ctx, SWEEPS, sh.ordered_allreduce(dist))
    out[rank] = (c.factors().tobytes(), c.x().astype(np.float64).tobytes(), st)
    c.close()
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("exec_path", ["graph", "persistent"])
@pytest.mark.parametrize("dims,edge", [
    ((14, 12, 10, 9), {(0, 1): 3, (0, 2): 4, (0, 3): 2, (1, 2): 3, (1, 3): 2, (2, 3): 3}),
    ((21, 18, 16), {(0, 1): 3, (0, 2): 2, (1, 2): 4}),
])
def test_two_slabs_match_the_whole_problem(dims, edge, exec_path):
    from paper_2511_16358_gb300 import binding as b
    case = make_case(dims, edge, 0.35, seed=491, kind="max1", sigma=0.02)
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, _free_port(), case, b.FP64, exec_path, out), nprocs=world,
                           join=True, start_method="spawn")
        res = dict(out)
    R = case["R"]
    bounds = [sh.slab_bounds(dims[0], world, r) for r in range(world)]
    slabs, xs = [], []
    for r, (lo, hi) in enumerate(bounds):
        g, x, st = res[r]
        slabs.append(np.frombuffer(g))
        xs.append(np.frombuffer(x).reshape((hi - lo,) + tuple(dims[1:])))
    # the factors the slabs share are the same bits on both processes
    from paper_2511_16358_gb300 import inputs as inp
    F = [inp.unpack_factors(s, (hi - lo,) + tuple(dims[1:]), R) for s, (lo, hi) in zip(slabs, bounds)]
    for k in range(1, len(dims)):
        for l in range(len(dims)):
            if l != k:
                assert F[0][(k, l)].tobytes() == F[1][(k, l)].tobytes()
    G, X = case["G0"].copy(), case["X0"].copy()
    log = oracle.complete(dims, R, 0.1, G, X, case["mask"], max_sweeps=SWEEPS)
    assert rel_err(sh.merge_factors(slabs, dims, R, bounds), G) < 1e-10
    assert rel_err(np.concatenate(xs, axis=0), X) < 1e-10
    st = res[0][2]
    assert st["sweeps_done"] == SWEEPS
    for key in ("sweeps_done", "rel_change", "objective"):  # rse / rmse are NaN without a truth
        assert res[1][2][key] == st[key]
    assert st["rel_change"] == pytest.approx(log[-1]["rel_change"], rel=1e-9)
    assert st["objective"] == pytest.approx(log[-1]["objective"], rel=1e-9)
