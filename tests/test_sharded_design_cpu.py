"""The multi-GPU slab-sharding design, checked on CPU with two gloo ranks.

The library runs on one GPU; sharding is a design (X split into slabs along
its largest mode p).  This test carries that design out in plain numpy on two
gloo ranks and checks that its exchanges are enough to reproduce one sweep of
Algorithm 1 exactly:

  * mode k != p: each rank contracts its slab, M_k partials are summed by one
    all-reduce (I_k x Q_k values); K_k = Z_k^T Z_k needs factors only and is
    formed redundantly on every rank;
  * mode p: rows j of M_p are slab-local, so each rank solves its own columns
    of G_{p,.} and the columns are all-gathered;
  * the X update is slab-local; the stop-test sums need one scalar all-reduce.

Every block uses the regrouped systems H = E_j^T K_k E_j + rho I,
b = E_j^T M_k(j,:)^T + rho g_old (Prop. 1 with eq. (updateG)).  After one
sweep both ranks hold bitwise-equal factors, and factors and tensor equal the
FP64 oracle's within 1e-10.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

RHO = 0.1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _slab(n, rank, world):
    return n * rank // world, n * (rank + 1) // world


def _all_gather_slabs(local, axis, n, world):
    """All-gather of slabs along ``axis`` whose widths differ by rank (gloo
    wants equal sizes: each slab is padded to the widest, then trimmed)."""
    width = max(b - a for a, b in (_slab(n, r, world) for r in range(world)))
    pad = [(0, 0)] * local.ndim
    pad[axis] = (0, width - local.shape[axis])
    parts = [torch.zeros([width if d == axis else local.shape[d] for d in range(local.ndim)],
                         dtype=torch.float64) for _ in range(world)]
    dist.all_gather(parts, torch.from_numpy(np.ascontiguousarray(np.pad(local, pad))))
    keep = []
    for r, t in enumerate(parts):
        a, b = _slab(n, r, world)
        keep.append(np.take(t.numpy(), np.arange(b - a), axis=axis))
    return np.concatenate(keep, axis=axis)


def _recon(dims, R, F, index_ranges):
    """prod_{p<q} W_{p,q}(i_p, i_q) over the given index range of every mode."""
    N = len(dims)
    X = np.ones([hi - lo for lo, hi in index_ranges])
    for p in range(N):
        for q in range(p + 1, N):
            W = F[(p, q)].T @ F[(q, p)]
            lp, hp = index_ranges[p]
            lq, hq = index_ranges[q]
            shp = [1] * N
            shp[p], shp[q] = hp - lp, hq - lq
            X = X * W[lp:hp, lq:hq].reshape(shp)
    return X


def _rank(rank, world, port, case, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2511_16358_gb300 import inputs as inp
    from tests.test_oracle_pins import _E, _prop1_Z, _unfold_littleendian

    dims, R = case["dims"], case["R"]
    N = len(dims)
    p = int(np.argmax(dims))
    lo, hi = _slab(dims[p], rank, world)
    take = [slice(None)] * N
    take[p] = slice(lo, hi)
    Xs = case["X0"][tuple(take)].copy()                 # this rank's slab of X
    ms = case["mask"][tuple(take)].astype(bool)
    G = case["G0"].copy()
    F = inp.unpack_factors(G, dims, R)

    for k in range(N):
        Z = _prop1_Z(dims, R, F, k)                     # factors only: the same on every rank
        K = Z.T @ Z
        if k != p:
            # rows of Z_k (little-endian over the modes other than k) that fall in this slab
            rest = [m for m in range(N) if m != k]
            idx = np.indices([dims[m] for m in rest]).reshape(len(rest), -1, order="F")
            rows = (idx[rest.index(p)] >= lo) & (idx[rest.index(p)] < hi)
            Mpart = _unfold_littleendian(Xs, k) @ Z[rows]
            M = torch.from_numpy(np.ascontiguousarray(Mpart))
            dist.all_reduce(M)                          # the one data exchange of mode k
            M = M.numpy()
            js = range(dims[k])
        else:
            M = np.zeros((dims[k], Z.shape[1]))
            M[lo:hi] = _unfold_littleendian(Xs, k) @ Z  # slab-local rows of M_p
            js = range(lo, hi)
        for i in range(N):
            if i == k:
                continue
            for j in js:
                E = _E(dims, R, F, k, i, j)
                H = E.T @ K @ E + RHO * np.eye(E.shape[1])
                b = E.T @ M[j] + RHO * F[(k, i)][:, j]
                F[(k, i)][:, j] = np.linalg.solve(H, b)
        if k == p:
            # all-gather the updated columns of every G_{p,.}
            for i in range(N):
                if i == k:
                    continue
                F[(k, i)][:, :] = _all_gather_slabs(F[(k, i)][:, lo:hi], 1, dims[p], world)

    ranges = [(0, d) for d in dims]
    ranges[p] = (lo, hi)
    rec = _recon(dims, R, F, ranges)
    Xn = np.where(ms, Xs, (rec + RHO * Xs) / (1 + RHO))
    sums = torch.tensor([np.sum((Xn - Xs) ** 2), np.sum(Xs ** 2)], dtype=torch.float64)
    dist.all_reduce(sums)                               # scalar exchange of the stop test
    Gs = [torch.zeros(G.size, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(Gs, torch.from_numpy(G))
    Xall = _all_gather_slabs(Xn, p, dims[p], world)
    if rank == 0:
        out["G"] = [g.numpy() for g in Gs]
        out["X"] = Xall
        out["rel_change"] = float(np.sqrt(sums[0] / sums[1]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("dims,edge", [
    ((8, 5, 4), {(0, 1): 2, (0, 2): 3, (1, 2): 2}),
    ((3, 7, 4, 2), {(0, 1): 2, (0, 2): 1, (0, 3): 2, (1, 2): 3, (1, 3): 2, (2, 3): 2}),
])
def test_two_rank_slab_sharded_sweep_equals_oracle(dims, edge):
    import oracle
    from tests._cases import make_case
    case = make_case(dims, edge, 0.5, seed=sum(dims) + 300)
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), case, out), nprocs=world, join=True)
        res = dict(out)
    G, X = case["G0"].copy(), case["X0"].copy()
    st = oracle.sweep(dims, case["R"], RHO, G, X, case["mask"])
    assert np.array_equal(res["G"][0], res["G"][1])     # bitwise-equal replicas of the factors
    den = np.max(np.abs(G))
    assert np.max(np.abs(res["G"][0] - G)) < 1e-10 * den
    assert np.max(np.abs(res["X"] - X)) < 1e-10 * np.max(np.abs(X))
    assert abs(res["rel_change"] - st["rel_change"]) < 1e-9 * st["rel_change"]
