"""Build libgs.so (the CUDA library behind include/gs.h) in-tree for sm_103a, and its bounds-checked
twin libgs_checked.so (the same sources compiled with GS_CHECKED=1: data-dependent indices are
compared with their buffers' lengths and violations recorded instead of followed).

Each translation unit under csrc/ is compiled by its own nvcc process (in parallel), then linked
into paper_2605_10760_gb300/_build/ with the CUDA runtime linked statically.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libgs.so")
VARIANTS = {"release": ("libgs.so", []), "checked": ("libgs_checked.so", ["-DGS_CHECKED=1"])}
ARCH_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-DGS_ARCH=1030",
          "-I" + os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgs")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [os.path.join(ROOT, "include", "gs.h"),
                                                                          os.path.abspath(__file__)]


def _stamp(flags) -> str:
    h = hashlib.sha256()
    for p in _deps():
        with open(p, "rb") as f:
            h.update(p.encode() + f.read())
    h.update(" ".join(ARCH_FLAGS + COMMON + list(flags)).encode())
    return h.hexdigest()


def _compile(nvcc: str, src: str, obj: str, flags, verbose: bool) -> str:
    cmd = [nvcc, *ARCH_FLAGS, *COMMON, *flags, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
    if verbose and r.stderr:
        sys.stderr.write(r.stderr)
    return obj


def build(force: bool = False, verbose: bool = False, extra=(), variant: str | None = None) -> str:
    """Compile (if its sources changed) each variant, or only `variant`: every translation unit of
    every variant in one pool of nvcc processes, then one link per variant.  Returns the path of
    the release library (or of `variant`'s)."""
    os.makedirs(OUT, exist_ok=True)
    names = [variant] if variant else list(VARIANTS)
    todo = {}
    for v in names:
        lib_name, vflags = VARIANTS[v]
        flags = list(vflags) + list(extra)
        lib = os.path.join(OUT, lib_name)
        stamp = _stamp(flags)
        stamp_file = lib + ".stamp"
        if force or not (os.path.exists(lib) and os.path.exists(stamp_file) and open(stamp_file).read() == stamp):
            todo[v] = (lib, flags, stamp)
    if todo:
        nvcc = _nvcc()
        with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as pool:
            jobs = {}
            for v, (lib, flags, _) in todo.items():
                tag = os.path.splitext(os.path.basename(lib))[0]
                jobs[v] = [pool.submit(_compile, nvcc, src, os.path.join(OUT, "%s.%s.o" % (tag, os.path.basename(src))),
                                       flags, verbose) for src in _sources()]
            objs = {v: [f.result() for f in fs] for v, fs in jobs.items()}
        for v, (lib, flags, stamp) in todo.items():
            tmp = lib + ".tmp"
            cmd = [nvcc, *ARCH_FLAGS, "-shared", "-cudart", "static", *objs[v], "-o", tmp]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
            os.replace(tmp, lib)
            with open(lib + ".stamp", "w") as f:
                f.write(stamp)
    return os.path.join(OUT, VARIANTS[variant or "release"][0])


if __name__ == "__main__":
    extra = [a for a in sys.argv[1:] if a.startswith("-X")]
    print(build(force="--force" in sys.argv, verbose=True, extra=extra))
