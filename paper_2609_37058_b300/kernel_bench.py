"""Kernel-level driver: runs one library kernel entry point on a seeded batch.

    python -m paper_2609_37058_b300.kernel_bench --op mixed --batch 148 --b 256 --reps 2

Ops: ``mixed`` (six-slice double-float GEMM), ``hp`` (seven-slice FP64-class
GEMM), ``f64`` (FP64 CUDA-core GEMM), ``inv64`` / ``inv32`` (batched
Gauss-Jordan inverses).  Each repetition is one call of the C entry point
(host buffers in and out).  The call prints one JSON line with the wall time
per call and the largest deviation from numpy's own product or inverse, so
that the command is a self-checking target for profilers.

``--op kpm`` runs the KPM moments kernel on a seeded junction of
``--layers`` layers of block size ``--b`` with ``--batch`` random-phase
vectors and ``--moments`` moments (one launch); its self-check is that
mu_0 equals the matrix size and no |mu_n| exceeds it.

``--op peaks`` measures the roofline denominators that the box's measured
peak file does not hold: the library's FP64 and FP32 FMA-loop probes
(``rgf_peak_fma``, best of several launches), and, for comparison, cuBLAS
through torch: FP64 DGEMM and TF32 GEMM (fp32 inputs with TF32 tensor-core
math allowed) of 8192^3, best of 5 after warm-up, CUDA events.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import rgf


def _inputs(op: str, batch: int, b: int, seed: int):
    rng = np.random.default_rng(seed)

    def cplx(shape):
        return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)

    if op in ("inv64", "inv32"):
        # Diagonally weighted so that every matrix is well conditioned.
        A = cplx((batch, b, b)) / np.sqrt(b) + 2.0 * np.eye(b)
        return (A,)
    return cplx((batch, b, b)), cplx((batch, b, b))


def run(op: str, batch: int, b: int, reps: int, seed: int = 0) -> dict:
    args = _inputs(op, batch, b, seed)
    fn = {
        "mixed": lambda: rgf.rgf_kernel_zgemm_mixed(*args, core=0),
        "hp": lambda: rgf.rgf_kernel_zgemm_hp(*args),
        "f64": lambda: rgf.rgf_kernel_zgemm_f64(*args),
        "inv64": lambda: rgf.rgf_kernel_inverse_f64(*args)[0],
        "inv32": lambda: rgf.rgf_kernel_inverse_c64(args[0].astype(np.complex64))[0],
    }[op]
    out = None
    t0 = time.perf_counter()
    for _ in range(reps):
        out = fn()
    dt = (time.perf_counter() - t0) / max(reps, 1)
    if op in ("inv64", "inv32"):
        dev = float(np.abs(np.matmul(args[0], out.astype(np.complex128)) - np.eye(b)).max())
        what = "max |A X - I|"
    else:
        dev = float(np.abs(out - np.matmul(*args)).max())
        what = "max |C - A B|"
    return {"op": op, "batch": batch, "b": b, "reps": reps, "s_per_call": dt, "check": what, "value": dev}


def kpm_run(layers: int, b: int, n_vec: int, n_mom: int, seed: int) -> dict:
    from synth import random_device
    from synth.devices import random_phase_vectors
    dev = random_device(layers, b, seed, metal_frac=0.25, gap_offset=0.6)
    n = layers * b
    R = random_phase_vectors(n_vec, n, seed + 1)
    with rgf.KPM(dev) as k:
        alpha, beta = k.scale(random_phase_vectors(1, n, seed + 2)[0], 50, 0.1)
        t0 = time.perf_counter()
        mu = k.moments(R, n_mom, alpha, beta)
        dt = time.perf_counter() - t0
    return {"op": "kpm", "layers": layers, "b": b, "vectors": n_vec, "moments": n_mom, "s_per_call": dt,
            "mu0_error": float(abs(mu[0] - n)), "max_abs_mu_over_mu0": float(np.abs(mu).max() / mu[0])}


def peaks(reps: int = 5) -> dict:
    import torch
    out = {}
    for kind, name in ((0, "fp64_fma_tflops"), (1, "fp32_fma_tflops")):
        rgf.rgf_peak_fma(kind, 8, 1 << 12)
        out[name] = max(rgf.rgf_peak_fma(kind, 8, 1 << 16)[0] for _ in range(reps))

    def gemm_tflops(dtype, n, tf32):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        a = torch.randn(n, n, device="cuda", dtype=dtype)
        b = torch.randn(n, n, device="cuda", dtype=dtype)
        for _ in range(2):
            torch.matmul(a, b)
        best = 0.0
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            e1.synchronize()
            best = max(best, 2.0 * n ** 3 / (e0.elapsed_time(e1) * 1e-3) / 1e12)
        torch.backends.cuda.matmul.allow_tf32 = False
        return best

    out["fp64_dgemm_cublas_tflops"] = gemm_tflops(torch.float64, 8192, False)
    out["tf32_gemm_cublas_tflops"] = gemm_tflops(torch.float32, 8192, True)
    out["fp32_gemm_cublas_tflops"] = gemm_tflops(torch.float32, 8192, False)
    out["device"] = torch.cuda.get_device_name()
    return out


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--op", choices=["mixed", "hp", "f64", "inv64", "inv32", "peaks", "kpm"], default="mixed")
    ap.add_argument("--batch", type=int, default=148)
    ap.add_argument("--b", type=int, default=256)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--layers", type=int, default=40, help="layers of the kpm op's junction")
    ap.add_argument("--moments", type=int, default=16, help="moments of the kpm op")
    a = ap.parse_args(argv)
    if a.op == "peaks":
        print(json.dumps(peaks()))
        return 0
    if a.op == "kpm":
        res = kpm_run(a.layers, a.b, a.batch, a.moments, a.seed)
        print(json.dumps(res))
        return 0 if res["mu0_error"] == 0.0 and res["max_abs_mu_over_mu0"] <= 1.0 + 1e-9 else 1
    res = run(a.op, a.batch, a.b, a.reps, a.seed)
    print(json.dumps(res))
    limit = {"mixed": 1e-9, "hp": 1e-12, "f64": 1e-12, "inv64": 1e-10, "inv32": 1e-3}[a.op]
    return 0 if res["value"] <= limit * max(1.0, np.sqrt(a.b)) else 1


if __name__ == "__main__":
    raise SystemExit(main())
