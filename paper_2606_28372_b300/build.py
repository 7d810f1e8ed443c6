"""Builds libcatune.so in-tree for sm_103a with nvcc (no JIT, no torch extension cache).

Each source compiles to its own object under `_build/` (in parallel, one nvcc per source), then
one link makes the shared library.  A source is recompiled when it or any header is newer than
its object."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "..", "_build")
LIB = os.path.join(HERE, "libcatune.so")
SOURCES = ["space.cu", "search.cu", "rules.cu", "optim.cu", "batch.cu", "surrogate.cu", "noalloc.cu", "measure.cu", "scan_lut.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-Xcompiler", "-fPIC"]


def sources():
    return [os.path.join(CSRC, s) for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]


def headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".hpp"))]
    hs.append(os.path.join(HERE, "..", "include", "catune.h"))
    return hs


def _obj(src):
    return os.path.join(OBJ, os.path.basename(src)[:-3] + ".o")


def _stale_objects():
    newest_header = max(os.path.getmtime(h) for h in headers())
    out = []
    for s in sources():
        o = _obj(s)
        if not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), newest_header):
            out.append(s)
    return out


def stale() -> bool:
    if not os.path.exists(LIB) or _stale_objects():
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(_obj(s)) > t for s in sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not stale():
        return LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    os.makedirs(OBJ, exist_ok=True)
    todo = sources() if force else _stale_objects()
    ptxas = ["-Xptxas", "-v" if verbose else "-O3"]

    def compile_one(src):
        tmp = _obj(src) + f".tmp{os.getpid()}"
        subprocess.check_call([nvcc, *ARCH, *FLAGS, *ptxas, "-c", "-o", tmp, src])
        os.replace(tmp, _obj(src))

    with ThreadPoolExecutor(max_workers=max(1, min(len(todo), os.cpu_count() or 1))) as ex:
        list(ex.map(compile_one, todo))
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc, *ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", tmp, *[_obj(s) for s in sources()]])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv))
