"""The allocation-free reconstruction entry point.

ifctn_reconstruct_noalloc serves callers that cannot call cudaMalloc (their
device memory belongs to another allocator, or an allocation would stall their
path): it keeps its scratch in a fixed array inside the library.  This test
calls it twice in a row, through the C ABI, and checks each result against the
context-based ifctn_reconstruct and against the FP64 oracle's reconstruction, within the
tolerances the other tests use.
It lives in its own file, collected last, and must pass alone or after the
rest of the suite.
"""
import numpy as np
import pytest

import oracle
from paper_2511_16358_gb300 import binding as b
from paper_2511_16358_gb300 import inputs as inp

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [(b.FP64, 1e-13), (b.MIXED, 2e-6)])
def test_noalloc_reconstruct_matches_reconstruct_twice(precision, tol):
    import torch
    dims = (23, 17, 12, 9)
    R = inp.rank_matrix(4, {(0, 1): 3, (0, 2): 2, (0, 3): 4, (1, 2): 2, (1, 3): 1, (2, 3): 3})
    G = inp.gaussian_factors(dims, R, 424242)
    dt = b.tensor_dtype(precision)
    P = int(np.prod(dims))
    c = b.Completion(dims, R, np.zeros(P, dtype=dt), np.zeros(P, dtype=np.uint8), precision=precision,
                     init_factors=G.copy(), max_sweeps=1, tol=0.0)
    ref = c.reconstruct()
    c.close()
    truth = oracle.reconstruct(dims, R, G)
    Gd = torch.from_numpy(G).cuda()
    tdt = torch.float64 if precision == b.FP64 else torch.float32
    for _ in range(2):
        out = torch.full(dims, float("nan"), dtype=tdt, device="cuda")
        b.reconstruct_noalloc(dims, R, precision, Gd, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
        assert err < tol, err
        err_o = np.max(np.abs(got - truth)) / np.max(np.abs(truth))
        assert err_o < tol, err_o


def test_noalloc_rejects_oversized_and_host_buffers():
    import torch
    dims = (2048, 2048)  # pair matrix of 4M entries: above the 8 MiB array in FP64
    R = inp.rank_matrix(2, 2)
    G = torch.zeros(inp.factor_size(dims, R), dtype=torch.float64, device="cuda")
    out = torch.zeros(dims, dtype=torch.float64, device="cuda")
    with pytest.raises(b.IfctnError) as ei:
        b.reconstruct_noalloc(dims, R, b.FP64, G, out)
    assert ei.value.status == b.EINVAL and "scratch" in b.last_error()
    small = (8, 7)
    Gh = torch.zeros(inp.factor_size(small, R), dtype=torch.float64)
    outd = torch.zeros(small, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):  # the binding refuses host memory
        b.reconstruct_noalloc(small, R, b.FP64, Gh, outd)
    # and so does the library itself, for a caller that goes around the binding
    import ctypes
    d = (ctypes.c_int64 * 4)(8, 7, 0, 0)
    r = (ctypes.c_int32 * 16)(*([0, 2, 0, 0, 2, 0] + [0] * 10))
    rc = b.load().ifctn_reconstruct_noalloc(2, d, r, b.FP64, ctypes.c_void_p(Gh.data_ptr()),
                                            ctypes.c_void_p(outd.data_ptr()), None)
    assert rc == b.EINVAL and "current device" in b.last_error()
