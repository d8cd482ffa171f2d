"""Extended-precision (x87 80-bit) oracle: ctypes binding of ``rgf_ext.c``.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, the golden-value script beside
them, ``__graft_entry__`` (its build step compiles the C file) and the
CPU-baseline leg of ``bench.py`` may import this module.  The CUDA library
never calls it and shares no code with it.

``transmission`` evaluates the same textbook steps as ``rgf_oracle`` (Sancho-
Rubio leads refined by Newton steps on their fixed-point equation, Sigma and
Gamma, left-to-right sweep, Caroli trace) with every real number a
64-bit-significand ``long double``; energies run in parallel on
the host cores.  It is pinned in ``tests/test_oracle_ext.py`` (mpmath dense
inversion at 40 digits, the uniform-chain closed form in mpmath, the FP64
oracle on well-conditioned energies).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rgf_ext.c")
LIB = os.path.join(HERE, "_rgf_ext.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile ``rgf_ext.c`` into ``_rgf_ext.so`` (gcc, OpenMP over energies).
    No fast-math: the rounding of every long double operation is IEEE's."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        lib.rgf_ext_transmission.argtypes = [
            ctypes.c_int, ctypes.c_int, dp, dp, dp, dp,
            ctypes.POINTER(dp), ctypes.POINTER(dp), dp, ctypes.c_int, ctypes.c_double,
            ctypes.c_double, ctypes.c_int, ctypes.c_int, dp, dp, ctypes.POINTER(ctypes.c_int)]
        lib.rgf_ext_transmission.restype = None
        lib.rgf_ext_surface_gf.argtypes = [
            ctypes.c_int, ctypes.POINTER(dp), ctypes.c_int, ctypes.c_double, ctypes.c_double,
            ctypes.c_double, ctypes.c_int, ctypes.c_int, dp, dp]
        lib.rgf_ext_surface_gf.restype = ctypes.c_int
        _lib = lib
    return _lib


def _c128(x):
    return np.ascontiguousarray(x, dtype=np.complex128)


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _lead_ptrs(lead, keep):
    arrs = [_c128(getattr(lead, k)) for k in ("H00", "S00", "H10", "S10", "Hc", "Sc")]
    keep.extend(arrs)
    return (ctypes.POINTER(ctypes.c_double) * 6)(*[_ptr(a) for a in arrs])


def transmission(dev, energies, eta, tol=1e-18, max_iter=120, newton_steps=3, threads=None,
                 return_info=False):
    """T(E) in extended precision, rounded to float64 at the end.

    ``tol`` is the Sancho-Rubio stop (max(||alpha||, ||beta||) <= tol ||a||);
    its default sits just above the long double unit roundoff, so the
    decimation runs to the precision it carries.  ``newton_steps`` Newton
    steps on the fixed-point equation follow the decimation (0: none).  ``threads`` sets
    OMP_NUM_THREADS for this call's process if given before the first call.
    """
    if threads is not None:
        os.environ["OMP_NUM_THREADS"] = str(int(threads))
    lib = _load()
    E = np.ascontiguousarray(energies, dtype=np.float64)
    nE = E.shape[0]
    N, b = dev.n_layers, dev.b
    keep = []
    Hd, Sd = _c128(dev.H_diag), _c128(dev.S_diag)
    Hl = _c128(dev.H_lower) if N > 1 else np.zeros((1, b, b), np.complex128)
    Sl = _c128(dev.S_lower) if N > 1 else np.zeros((1, b, b), np.complex128)
    pL, pR = _lead_ptrs(dev.lead_L, keep), _lead_ptrs(dev.lead_R, keep)
    T = np.empty(nE)
    Ti = np.empty(nE)
    it = np.empty(2 * nE, dtype=np.int32)
    lib.rgf_ext_transmission(N, b, _ptr(Hd), _ptr(Sd), _ptr(Hl), _ptr(Sl), pL, pR, _ptr(E), nE,
                             float(eta), float(tol), int(max_iter), int(newton_steps), _ptr(T), _ptr(Ti),
                             it.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    if return_info:
        return T, dict(trace_imag=Ti, iters=it.reshape(nE, 2))
    return T


def surface_gf(lead, side, E, eta, tol=1e-18, max_iter=120, newton_steps=3):
    """Surface Green's function of one lead (side 'L' or 'R') as (hi, lo)
    complex128 pairs: hi + lo is the 80-bit result to about 2^-64.  Returns
    (hi, lo, iterations); iterations < 0 means not converged."""
    lib = _load()
    keep = []
    b = lead.H00.shape[0]
    p = _lead_ptrs(lead, keep)
    hi = np.empty((b, b), np.complex128)
    lo = np.empty((b, b), np.complex128)
    it = lib.rgf_ext_surface_gf(b, p, 1 if side == "R" else 0, float(E), float(eta), float(tol),
                                int(max_iter), int(newton_steps), _ptr(hi), _ptr(lo))
    return hi, lo, it
