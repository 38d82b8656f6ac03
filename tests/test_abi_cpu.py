"""CPU-side checks of the C ABI: the library builds, loads and exports every
entry point include/ifctn.h declares; arguments are validated before any GPU
work; the oracle and the CUDA path share no code."""
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ifctn.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2511_16358_gb300 import _build, binding
    _build.build()
    return binding.load()


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ifctn_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("ifctn_create", "ifctn_sweep", "ifctn_reconstruct", "ifctn_complete", "ifctn_submit",
              "ifctn_poll"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2511_16358_gb300 import binding
    so = binding.LIB_PATH
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (ifctn_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    assert set(binding.EXPORTED) == set(_declared())


def test_library_is_built_for_sm_103a(lib):
    from paper_2511_16358_gb300 import binding
    out = subprocess.run(["cuobjdump", "--list-elf", binding.LIB_PATH], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout


def _prob(**kw):
    from paper_2511_16358_gb300 import binding as b
    base = dict(dims=(4, 5, 6), ranks=np.full((3, 3), 2), rho=0.1, max_sweeps=3, tol=0.0,
                precision=b.FP64)
    base.update(kw)
    return b.make_problem(**base)


@pytest.mark.parametrize("bad", [
    dict(ranks=np.array([[0, 2, 2], [2, 0, 2], [2, 2, 0]]) * 0),
    dict(ranks=np.array([[0, 65, 2], [65, 0, 2], [2, 2, 0]])),  # above 64 at order 3
    dict(ranks=np.array([[0, 64, 65], [64, 0, 1], [65, 1, 0]])),  # Q_0 = 64 * 65 > 4096
    dict(dims=(4, 5, 6, 3), ranks=np.array([[0, 9, 2, 2], [9, 0, 2, 2], [2, 2, 0, 2], [2, 2, 2, 0]])),  # above 8 at order 4
    dict(dims=(4, 5), ranks=np.array([[0, 9], [9, 0]])),  # above 8 at order 2
    dict(ranks=np.array([[0, 2, 3], [2, 0, 2], [2, 2, 0]])),  # not symmetric
    dict(rho=0.0),
    dict(rho=-1.0),
    dict(rho=float("nan")),
    dict(rho=float("inf")),
    dict(tol=-1.0),
    dict(max_sweeps=-1),
    dict(dims=(4,)),
    dict(dims=(4, 0, 3)),
    dict(precision=7),
])
def test_invalid_problems_rejected_before_gpu_work(lib, bad):
    from paper_2511_16358_gb300 import binding as b
    dims = bad.get("dims", (4, 5, 6))
    n = int(np.prod([max(d, 1) for d in dims]))
    obs = np.zeros(n)
    mask = np.zeros(n, dtype=np.uint8)
    with pytest.raises(b.IfctnError) as ei:
        b.create(_prob(**bad), obs, mask)
    assert ei.value.status == b.EINVAL
    assert b.last_error()


def test_null_context_and_server_arguments(lib):
    from paper_2511_16358_gb300 import binding as b
    assert lib.ifctn_sweep(None, 1, None) == b.EINVAL
    assert lib.ifctn_poll(None, 1, None, None, 0) == b.EINVAL
    assert lib.ifctn_kernels_per_sweep(None) == 0
    lib.ifctn_destroy(None)
    lib.ifctn_server_destroy(None)


def test_server_and_noalloc_arguments_rejected_before_gpu_work(lib):
    import ctypes

    from paper_2511_16358_gb300 import binding as b
    srv = ctypes.c_void_p()
    assert lib.ifctn_server_create(0, 4, ctypes.byref(srv)) == b.EINVAL
    assert lib.ifctn_server_create(1 << 30, 0, ctypes.byref(srv)) == b.EINVAL
    assert lib.ifctn_submit(None, None, None, None, None, None) == b.EINVAL
    assert lib.ifctn_reconstruct_noalloc(3, None, None, 0, None, None, None) == b.EINVAL
    R2 = (ctypes.c_int32 * 16)(*([0, 2, 0, 0, 2, 0] + [0] * 10))
    dims = (ctypes.c_int64 * 4)(2048, 2048, 0, 0)
    host = np.zeros(8)
    hp = ctypes.c_void_p(host.ctypes.data)
    # pair matrices of 2048 x 2048 FP64 entries exceed the fixed scratch array: refused
    # from the sizes alone, before the buffers are looked at
    assert lib.ifctn_reconstruct_noalloc(2, dims, R2, b.FP64, hp, hp, None) == b.EINVAL
    assert "scratch" in b.last_error()
    R9 = (ctypes.c_int32 * 16)(*([0, 9, 0, 0, 9, 0] + [0] * 10))
    dims = (ctypes.c_int64 * 4)(4, 5, 0, 0)
    assert lib.ifctn_reconstruct_noalloc(2, dims, R9, b.FP64, hp, hp, None) == b.EINVAL


def test_noalloc_binding_refuses_mistyped_and_missized_buffers():
    """The allocation-free entry point takes no buffer lengths, so the binding
    refuses, before any call into the library, factors that are not FP64 or
    not exactly the packed size, and an output of the wrong dtype or size."""
    import torch

    from paper_2511_16358_gb300 import binding as b
    from paper_2511_16358_gb300 import inputs as inp
    dims = (5, 4, 3)
    R = inp.rank_matrix(3, 2)
    nf = inp.factor_size(dims, R)
    good_f = torch.zeros(nf, dtype=torch.float64)
    good_o = torch.zeros(dims, dtype=torch.float64)
    cases = [
        (torch.zeros(nf, dtype=torch.float32), good_o, "float64"),        # FP32 factors
        (torch.zeros(nf - 1, dtype=torch.float64), good_o, "elements"),  # short factors
        (good_f, torch.zeros((5, 4, 2), dtype=torch.float64), "elements"),  # mis-shaped out
        (good_f, torch.zeros(dims, dtype=torch.float32), "float64"),     # out dtype vs FP64
        (good_f, torch.zeros(60, dtype=torch.float64)[::1].view(5, 12).t(), "contiguous"),
        (np.zeros(nf), good_o, "torch tensor"),                          # host numpy buffer
        (good_f, good_o, "CUDA memory"),                                 # right sizes, host memory
    ]
    for f, o, word in cases:
        with pytest.raises(ValueError, match=word):
            b.reconstruct_noalloc(dims, R, b.FP64, f, o)
    with pytest.raises(ValueError, match="float32"):
        b.reconstruct_noalloc(dims, R, b.MIXED, good_f, good_o)


def test_oracle_and_cuda_path_share_no_code():
    pkg = os.path.join(ROOT, "paper_2511_16358_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, re.M), f
                assert "ifctn_oracle" not in src and "ifo_" not in src, f
    # and the oracle uses nothing of the package or the CUDA library
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c", ".h")):
            src = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_2511_16358_gb300" not in src and "libifctn.so" not in src, f
            assert not re.search(r"#include\s*[<\"]cuda|^\s*(import|from)\s+(torch|cupy)\b", src, re.M), f
    osrc = open(os.path.join(ROOT, "oracle", "ifctn_oracle.c")).read()
    assert "#include \"" not in osrc  # only system headers
    opy = open(os.path.join(ROOT, "oracle", "__init__.py")).read()
    assert "paper_2511_16358_gb300" not in opy


def test_binding_refuses_non_contiguous_buffers():
    """The library takes plain pointers with C-order layouts: a strided view
    would be read as the wrong elements, so the binding refuses it."""
    import torch

    from paper_2511_16358_gb300 import binding as b
    a = np.zeros((4, 6))
    assert b.ptr(a) == a.ctypes.data and b.ptr(None) is None
    with pytest.raises(ValueError):
        b.ptr(a[:, ::2])
    with pytest.raises(ValueError):
        b.ptr(np.zeros((4, 6)).T)
    with pytest.raises(ValueError):
        b.ptr(torch.zeros(4, 6).t())
    with pytest.raises(TypeError):
        b.ptr([1.0, 2.0])
