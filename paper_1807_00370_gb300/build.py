"""Build the CUDA library libcrsolve.so in-tree (nvcc, sm_103a only).

Every translation unit under csrc/ is compiled in parallel with
``-gencode arch=compute_103a,code=sm_103a`` and linked into
``_build/libcrsolve.so``; the C ABI is declared in ``include/crsolve.h``.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libcrsolve.so")
# the same sources with every kernel index checked against the level sizes
DEBUG_LIB = os.path.join(BUILD, "libcrsolve_debug.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    cand = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    p = os.path.join(cand, "bin", "nvcc")
    return p if os.path.exists(p) else "nvcc"


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)]


def is_stale(debug: bool = False) -> bool:
    lib = DEBUG_LIB if debug else LIB
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in _deps())


def _variants(debug):
    """(library, object directory, extra flags) of the builds to run."""
    out = [(LIB, BUILD, [])]
    if debug:
        out.append((DEBUG_LIB, os.path.join(BUILD, "debug"), ["-DCRSOLVE_DEBUG_BOUNDS"]))
    return out


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile and link libcrsolve.so (and with debug=True also the
    bounds-checked libcrsolve_debug.so) if any source is newer (or force).
    All translation units of both libraries compile in parallel."""
    todo = [v for v in _variants(debug) if force or is_stale(v[0] == DEBUG_LIB)]
    if not todo:
        return LIB
    nvcc = _nvcc()
    procs, links = [], []
    for lib, odir, extra in todo:
        os.makedirs(odir, exist_ok=True)
        objs = []
        for src in _sources():
            obj = os.path.join(odir, os.path.basename(src)[:-3] + ".o")
            objs.append(obj)
            cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        links.append((lib, objs))
    failed = []
    for src, pr in procs:
        out, _ = pr.communicate()
        if pr.returncode != 0:
            failed.append((src, out.decode(errors="replace")))
    if failed:
        msg = "\n".join(f"--- {s}\n{o}" for s, o in failed)
        raise RuntimeError(f"nvcc failed:\n{msg}")
    for lib, objs in links:
        tmp = lib + f".{os.getpid()}.tmp"
        subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], check=True)
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, debug="--debug" in sys.argv))
