"""Build the RGF CUDA library in-tree for sm_103a.

``python -m paper_2609_37058_b300.build`` (or ``build()``) compiles every
``csrc/*.cu`` with nvcc into ``paper_2609_37058_b300/librgf.so``.  The
shared library is the product; the Python binding loads it with ctypes.
``build(debug=True)`` (``-d``) compiles the same sources with -DRGF_DEBUG
into ``librgf_debug.so`` (device-side index checks; see rgf_debug_flags).
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "librgf.so")
OUT_DEBUG = os.path.join(HERE, "librgf_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def build(verbose: bool = False, force: bool = False, extra=None, debug: bool = False) -> str:
    lib_out = OUT_DEBUG if debug else OUT
    extra = list(extra or []) + (["-DRGF_DEBUG"] if debug else [])
    srcs = sources()
    deps = srcs + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(os.path.dirname(HERE), "include", "*.h"))
    if not force and os.path.exists(lib_out):
        t = os.path.getmtime(lib_out)
        if all(os.path.getmtime(d) <= t for d in deps):
            return lib_out
    objdir = os.path.join(HERE, "_build_debug" if debug else "_build")
    os.makedirs(objdir, exist_ok=True)
    objs = []
    procs = []
    for s in srcs:
        o = os.path.join(objdir, os.path.basename(s) + ".o")
        cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               "-Xptxas", "-v" if verbose else "-O3", "-I", os.path.join(os.path.dirname(HERE), "include"),
               "-c", s, "-o", o] + list(extra or [])
        procs.append((s, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(o)
    failed = False
    for s, pr in procs:
        out, _ = pr.communicate()
        if pr.returncode != 0 or verbose:
            sys.stderr.write(out.decode(errors="replace"))
        if pr.returncode != 0:
            failed = True
    if failed:
        raise RuntimeError("nvcc failed")
    cmd = [nvcc(), *ARCH, "-shared", "-o", lib_out + ".tmp", *objs]
    subprocess.check_call(cmd)
    os.replace(lib_out + ".tmp", lib_out)
    return lib_out


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv, debug="-d" in sys.argv))
