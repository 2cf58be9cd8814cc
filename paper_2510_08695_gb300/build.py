"""Builds libbpdc.so (the CUDA decoder and its C-ABI) in-tree for sm_103a.

``python -m paper_2510_08695_gb300.build`` or ``build()``: every ``.cu`` file
under ``csrc/`` is compiled by nvcc in parallel, then linked into
``_build/libbpdc.so``; the same sources compiled with ``-DBPDC_CHECKS`` give
``_build/libbpdc_checked.so``, the bounds-checked debugging build (loaded
instead when the environment sets BPDC_CHECKED=1).  Rebuilds only when a
source or header is newer than the library.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libbpdc.so")
LIB_CHECKED = os.path.join(OUT, "libbpdc_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", f"-I{os.path.join(ROOT, 'include')}"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libbpdc.so")


def _inputs():
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    deps = srcs + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(ROOT, "include", "*.h"))
    return srcs, deps


def stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    _, deps = _inputs()
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in deps + [__file__])


def build(force: bool = False, verbose: bool = False) -> str:
    """Builds both libraries (all translation units of both in parallel)."""
    todo = [(lib, sub, extra) for lib, sub, extra in ((LIB, "", []), (LIB_CHECKED, "checked", ["-DBPDC_CHECKS"]))
            if force or stale(lib)]
    if not todo:
        return LIB
    nvcc = _nvcc()
    srcs, _ = _inputs()
    procs = []
    objs = {}
    for lib, sub, extra in todo:
        odir = os.path.join(OUT, sub)
        os.makedirs(odir, exist_ok=True)
        for s in srcs:
            o = os.path.join(odir, os.path.basename(s) + ".o")
            objs.setdefault(lib, []).append(o)
            cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", s, "-o", o]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append((s, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
    errors = []
    for s, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errors.append(f"{s}:\n{out}")
        elif verbose and out:
            print(out, file=sys.stderr)
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    for lib, _, _ in todo:
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.check_call([nvcc, *ARCH, "-shared", "-o", tmp, *objs[lib]])
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
