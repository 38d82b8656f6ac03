"""Builds libifctn.so (sm_103a) in-tree with nvcc, translation units in parallel."""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libifctn.so")
BUILD = os.path.join(HERE, "_build")
SOURCES = ["ifctn_persistent_f32.cu", "ifctn_persistent_f64.cu", "ifctn_contract_w_f32.cu",
           "ifctn_contract_w_f64.cu", "ifctn_kernels.cu", "ifctn_api.cu", "ifctn_server.cu", "ifctn_noalloc.cu",
           "ifctn_selftest.cu", "ifctn_xupdate.cu", "ifctn_wide.cu", "ifctn_plan.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-I" + os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _includes(path, seen):
    """The in-tree files `path` includes (#include "..."), transitively."""
    import re
    if path in seen:
        return
    seen.add(path)
    with open(path) as f:
        for name in re.findall(r'^\s*#\s*include\s+"([^"]+)"', f.read(), re.M):
            dep = os.path.normpath(os.path.join(os.path.dirname(path), name))
            if os.path.exists(dep):
                _includes(dep, seen)


def _sources_digest() -> str:
    """Digest of every library source and the public header (the tuning
    cache keys carry it, so a changed library never reuses stale choices)."""
    h = hashlib.sha256()
    for name in sorted(os.listdir(CSRC)):
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(name.encode() + f.read())
    with open(os.path.join(ROOT, "include", "ifctn.h"), "rb") as f:
        h.update(f.read())
    return h.hexdigest()[:16]


def _tu_flags(src):
    if src == "ifctn_api.cu":
        return [f'-DIFCTN_SOURCE_DIGEST="{_sources_digest()}"']
    return []


def _tu_digest(src) -> str:
    """Digest of one translation unit: its source, every in-tree header it
    includes and the compiler flags."""
    seen = set()
    _includes(os.path.join(CSRC, src), seen)
    h = hashlib.sha256()
    for path in sorted(seen):
        with open(path, "rb") as f:
            h.update(os.path.relpath(path, ROOT).encode() + f.read())
    h.update(" ".join(ARCH + FLAGS + _tu_flags(src)).encode())
    return h.hexdigest()


def _digest() -> str:
    h = hashlib.sha256()
    for src in SOURCES:
        h.update(_tu_digest(src).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles the translation units whose sources or headers changed (each
    object keeps the digest it was built from) and links libifctn.so."""
    stamp = os.path.join(BUILD, "stamp")
    dig = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == dig:
                return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()

    def comp(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        ostamp = obj + ".digest"
        d = _tu_digest(src)
        if not force and os.path.exists(obj) and os.path.exists(ostamp):
            with open(ostamp) as f:
                if f.read().strip() == d:
                    return obj
        cmd = [nvcc, *ARCH, *FLAGS, *_tu_flags(src), "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        with open(ostamp, "w") as f:
            f.write(d)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(comp, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(dig)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
