"""Host side of the slab-sharded sweep, on CPU: the slab cut and the factor
reassembly are inverse to each other, and the ordered allreduce gives every
gloo rank the same bits -- the sum in process order, also where the order of
floating-point additions changes the result."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2511_16358_gb300 import inputs as inp
from paper_2511_16358_gb300 import sharding as sh


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_slab_bounds_partition_the_first_mode():
    for I0 in (1, 5, 17, 288):
        for world in (1, 2, 3, 8):
            b = [sh.slab_bounds(I0, world, r) for r in range(world)]
            assert b[0][0] == 0 and b[-1][1] == I0
            assert all(b[r][1] == b[r + 1][0] for r in range(world - 1))
            assert max(h - l for l, h in b) - min(h - l for l, h in b) <= 1


def test_slab_factors_and_merge_are_inverse():
    dims = (11, 4, 5, 3)
    R = inp.rank_matrix(4, {(0, 1): 2, (0, 2): 3, (0, 3): 1, (1, 2): 2, (1, 3): 3, (2, 3): 2})
    G = inp.gaussian_factors(dims, R, 5)
    bounds = [sh.slab_bounds(11, 3, r) for r in range(3)]
    slabs = [sh.slab_factors(G, dims, R, lo, hi) for lo, hi in bounds]
    for (lo, hi), S in zip(bounds, slabs):
        F = inp.unpack_factors(S, (hi - lo,) + dims[1:], R)
        np.testing.assert_array_equal(F[(0, 2)], inp.unpack_factors(G, dims, R)[(0, 2)][:, lo:hi])
        np.testing.assert_array_equal(F[(2, 0)], inp.unpack_factors(G, dims, R)[(2, 0)])
    np.testing.assert_array_equal(sh.merge_factors(slabs, dims, R, bounds), G)


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # values whose sum depends on the order of the additions
    vals = np.array([[1e16, 1.0, 3.0], [1.0, -1e16, 0.5], [-1e16, 1e16, 0.25]][rank])
    sh.ordered_allreduce(dist)(vals)
    out[rank] = vals.tobytes()
    dist.barrier()
    dist.destroy_process_group()


def test_ordered_allreduce_same_bits_on_every_rank():
    world = 3
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = [np.frombuffer(out[r]) for r in range(world)]
    for r in range(1, world):
        assert res[r].tobytes() == res[0].tobytes()
    want = np.array([((1e16 + 1.0) + -1e16), ((1.0 + -1e16) + 1e16), (3.0 + 0.5) + 0.25])
    np.testing.assert_array_equal(res[0], want)
