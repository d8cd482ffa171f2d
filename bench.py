"""RGF transmission throughput benchmark (energy points per second).

Workload: the doped metal-semiconductor-metal junction with 500 principal
layers of block size 256 (2048 energies in [-1.5, 1.5] eV, eta = 1e-6,
synthetic seeded Hamiltonian).  One step = one wave of energies through the
whole path: decimation of both leads, self-energies, the 500-layer sweep and
the Caroli trace.  Ranks (torchrun) take disjoint energy waves; there is no
data-path collective.

Prints one JSON line.  See --help for the options.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "doped_N500_b256"
METRIC = "RGF energy-points/s (b=256, 500 layers), mixed vs FP64 at |dT|<=1e-6; p99 ms"
# ncu DRAM traffic of one slice-product GEMM launch (dram__bytes_read.sum +
# dram__bytes_write.sum), the BF16 flops of that launch, and the source it
# was measured on; reported (scaled by the flops of the timed launches) only
# while that source is unchanged.  Capture: batch 148, b = 256, tile 96
# (one launch under ncu).
GEMM_TRAFFIC = (700.945664e6 + 133.256192e6, 21 * 2.0 * 256 * 512 * 512 * 148,
                "f0230ed87ae0929900debefc3775a84e9e855f59737c52c103864abb3ea64a1a")


def parse():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--wave", type=int, default=512,
                    help="energies per step and rank (512: the 2048-energy grid in four full waves; larger waves "
                         "hide more of the seed inverse's panel latency, measured 45.6 / 47.4 / 48.2 / 48.3 "
                         "energies/s at 296 / 444 / 512 / 592)")
    ap.add_argument("--fp64-wave", type=int, default=148, help="energies of the timed FP64 GPU comparison wave")
    ap.add_argument("--no-compare", action="store_true", help="skip the FP64 GPU comparison step")
    ap.add_argument("--cpu-energies", type=int, default=2, help="energies of the oracle CPU sample")
    ap.add_argument("--batch-devices", type=int, default=64, help="devices of the uneven-batch run")
    ap.add_argument("--batch-energies", type=int, default=16,
                    help="energies per device of the uneven-batch run (0 skips it)")
    ap.add_argument("--serve-seconds", type=float, default=30.0, help="arrival window of the serving run (0 skips it)")
    ap.add_argument("--serve-rate", type=float, default=1.0, help="Poisson arrival rate of the serving run (1/s)")
    ap.add_argument("--serve-energies", default="32,128", help="energy-window sizes of serving requests (lo,hi)")
    ap.add_argument("--kpoints", type=int, default=8, help="k-points of the transverse-mesh run (0 skips it)")
    ap.add_argument("--ldos-energies", type=int, default=148, help="energies of the layer-DOS run (0 skips it)")
    ap.add_argument("--kpm-moments", type=int, default=256, help="Chebyshev moments of the KPM run (0 skips it)")
    ap.add_argument("--kpm-vectors", type=int, default=148, help="random vectors of the KPM run")
    ap.add_argument("--full-shapes", action="store_true",
                    help="also run the uneven-device batch at 512 energies per device and the Poisson "
                         "serving run at 200 requests/s (bounded window), plus a sustainable-rate point")
    ap.add_argument("--no-golden", action="store_true", help="skip the parity check at the stored oracle energies")
    ap.add_argument("--no-peaks", action="store_true", help="skip the FP64/FP32/TF32 peak probes")
    ap.add_argument("--parity-report", default="", help="write the per-energy parity table to this file")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.samples.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            try:
                sm.append(float(s[0]))
                mx = float(s[1])
            except ValueError:
                continue
            for n, v in zip(names, s[3:]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


def oracle_sample(dev, E, eta, n, info=False):
    """FP64 oracle on the first n energies; returns (T, seconds, threads)
    (and the per-energy decimation iteration counts when info is set)."""
    from oracle import rgf_oracle as o
    try:
        from threadpoolctl import threadpool_info
        threads = max((i.get("num_threads", 1) for i in threadpool_info()), default=1)
    except Exception:
        threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    T, inf = o.transmission(dev, E[:n], eta, return_info=True)
    dt = time.perf_counter() - t0
    if info:
        return T, dt, threads, [i["iters"] for i in inf]
    return T, dt, threads


def method_flop_per_energy(N, b, iters_L, iters_R):
    """Work of one energy point counted as the method's complex FP64
    operations (8 b^3 real flop per b x b x b product or inverse): the sweep
    (32 b^3 per layer after the first), g_0 (8 b^3), the decimation (56 b^3
    per iteration and lead), Sigma and Gamma (32 b^3) and G_{0,N-1} with the
    two trace products (24 b^3)."""
    b3 = float(b) ** 3
    return 32 * b3 * (N - 1) + 8 * b3 + 56 * b3 * (iters_L + iters_R) + 32 * b3 + 24 * b3


def golden_parity(rgf, plan_args, dev, report_path=""):
    """The mixed plan at the energies whose oracle values are stored with the
    tests (FP64 oracle and, when present, the extended-precision oracle):
    max |dT| against each, and the count above the 1e-6 bar.  Untimed."""
    import numpy as np
    base = os.path.join(ROOT, "tests", "golden", WORKLOAD)
    if not os.path.exists(base + ".txt"):
        return None
    g = np.loadtxt(base + ".txt")
    idx, Eg, To = g[:, 0].astype(int), g[:, 1], g[:, 2]
    Tx = None
    if os.path.exists(base + ".ext.txt"):
        x = np.loadtxt(base + ".ext.txt")
        if x.shape[0] == g.shape[0] and np.array_equal(x[:, 0].astype(int), idx):
            Tx = x[:, 2]
    with rgf.Plan(dev.n_layers, dev.b, **plan_args) as p:
        p.set_device(dev)
        T, err, fl = p.transmission(np.ascontiguousarray(Eg))
    d_o = np.abs(T - To)
    out = {"energies": int(len(idx)), "stride": int(idx[1] - idx[0]) if len(idx) > 1 else 1,
           "max_abs_dT_vs_fp64_oracle": float(d_o.max()), "over_1e-6_vs_fp64_oracle": int((d_o > 1e-6).sum()),
           "max_err_estimate": float(err.max())}
    if Tx is not None:
        d_x = np.abs(T - Tx)
        out.update({"max_abs_dT_vs_ext_oracle": float(d_x.max()), "over_1e-6_vs_ext_oracle": int((d_x > 1e-6).sum()),
                    "max_abs_fp64_oracle_vs_ext": float(np.abs(To - Tx).max())})
    if report_path:
        with open(report_path, "w") as f:
            f.write(f"# {WORKLOAD}: mixed path vs stored oracle values, every stored energy\n")
            f.write("# index E T_mixed err_estimate |dT|_vs_fp64_oracle |dT|_vs_ext_oracle flags\n")
            for k in range(len(idx)):
                dx = abs(T[k] - Tx[k]) if Tx is not None else float("nan")
                f.write(f"{idx[k]} {Eg[k]:.6f} {T[k]:.12e} {err[k]:.2e} {d_o[k]:.2e} {dx:.2e} {int(fl[k])}\n")
    return out


def tc_source_hash():
    import hashlib
    with open(os.path.join(ROOT, "paper_2609_37058_b300", "csrc", "tc_gemm.cu"), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def run_reference(args, rank, world):
    """The oracle, as it stands, on the host cores: each step is a bounded
    sample (one energy) of the same workload."""
    if rank != 0:
        return
    from synth import make_workload
    dev, E, eta = make_workload(WORKLOAD)
    times, threads = [], 1
    for k in range(args.warmup + args.steps):
        _, dt, threads = oracle_sample(dev, E[k % len(E):], eta, 1)
        if k >= args.warmup:
            times.append(dt)
    per = sum(times) / len(times)
    value = 1.0 / per
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "energy-points/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded junction Hamiltonian)",
        "config": {"workload": WORKLOAD, "n_layers": 500, "b": 256, "energies_per_step": 1, "eta": 1e-6},
        "cpu_baseline": {"value": value, "unit": "energy-points/s", "cores": threads, "kind": "oracle",
                         "sample": f"1 energy per step of {WORKLOAD}, numpy FP64 oracle"},
        "e2e": {"value": value, "unit": "energy-points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_batched(args, rgf):
    """Uneven devices through the server: N log-uniform in 50..1000 layers,
    b in {64, 96, 128, 192, 256, 320}, all submitted at once; energy
    points per second of wall time from the first submission to the last
    result.  (Parity of the server against the oracle is in the tests.)"""
    import numpy as np
    import torch

    from synth.gpu_devices import random_device_gpu, uneven_shapes

    shapes = uneven_shapes(args.batch_devices, 3, N_lo=50, N_hi=1000, b_choices=[64, 96, 128, 192, 256, 320])
    devs = [random_device_gpu(N, b, s, metal_frac=0.25, gap_offset=0.6) for N, b, s in shapes]
    nE = args.batch_energies
    E = np.linspace(-2.0, 2.0, nE)
    eta = 1e-5
    torch.cuda.synchronize()
    with rgf.Server(slots=148, class_step=32, tuning="default") as sv:
        t0 = time.perf_counter()
        tickets = [sv.submit(d, E, eta) for d in devs]
        res = [sv.poll(t, timeout_us=1_800_000_000) for t in tickets]
        wall = time.perf_counter() - t0
        st = sv.stats()
    if any(r is None for r in res):
        return {"error": "a request did not complete"}
    n_pts = nE * len(devs)
    del devs
    torch.cuda.empty_cache()
    Ns = [N for N, _, _ in shapes]
    return {"workload": "uneven_devices", "devices": len(shapes), "N_range": [min(Ns), max(Ns)],
            "N_mean": float(np.mean(Ns)), "b_set": sorted({b for _, b, _ in shapes}),
            "energies_per_device": nE, "eta": eta, "energy_points": n_pts, "seconds": wall,
            "value": n_pts / wall, "unit": "energy-points/s", "engines": st["engines"], "steps": st["steps"],
            "decimation_batches": st["decimations"], "fp64_reseeds": st["fp64_reseeds"],
            "workspace_bytes": st["workspace_bytes"], "peak_resident_bytes": st["peak_resident_bytes"],
            "flags_nonzero": int(sum(int(np.count_nonzero(r[2] & ~rgf.RGF_FLAG_REFINE)) for r in res)),
            "max_err_estimate": float(max(float(np.max(r[1])) for r in res))}


def run_serving(args, rgf):
    """Open-loop serving: Poisson arrivals, N log-uniform in 20..2000
    layers, b uniform in 96..288, energy windows of the given sizes; every
    request's device is drawn on the GPU before the clock starts and
    submitted at its arrival time.  Latency = submission to completion."""
    import numpy as np
    import torch

    from synth.devices import serving_trace
    from synth.gpu_devices import random_device_gpu

    lo, hi = (int(x) for x in args.serve_energies.split(","))
    trace = serving_trace(4, rate=args.serve_rate, duration=args.serve_seconds, N_lo=20, N_hi=2000, b_lo=96,
                          b_hi=288, nE_lo=lo, nE_hi=hi)
    devs = [random_device_gpu(r["N"], r["b"], r["seed"], metal_frac=0.25, gap_offset=0.6) for r in trace]
    torch.cuda.synchronize()
    with rgf.Server(slots=148, class_step=32, tuning="default") as sv:
        tickets = []
        t0 = time.perf_counter()
        for r, d in zip(trace, devs):
            delay = t0 + r["t"] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets.append(sv.submit(d, r["E"], r["eta"]))
        res = [sv.poll(t, timeout_us=1_800_000_000) for t in tickets]
        wall = time.perf_counter() - t0
        st = sv.stats()
    del devs
    torch.cuda.empty_cache()
    ok = [r for r in res if r is not None]
    n_pts = sum(r["n_E"] for r in trace)
    work = sum(r["n_E"] * r["N"] * r["b"] ** 3 * 32 for r in trace)  # sweep flop, 32 b^3 per layer
    return {"workload": "poisson_requests", "rate_per_s": args.serve_rate, "arrival_window_s": args.serve_seconds,
            "requests": len(trace), "completed": len(ok), "N_range": [20, 2000], "b_range": [96, 288],
            "energies_per_request": [lo, hi], "energy_points": n_pts, "seconds": wall,
            "energy_points_per_s": n_pts / wall if wall > 0 else None,
            "p50_ms": st["latency_p50_ms"], "p99_ms": st["latency_p99_ms"], "max_ms": st["latency_max_ms"],
            "engines": st["engines"], "peak_resident_bytes": st["peak_resident_bytes"],
            "capacity_note": "admission capped at min(150 GB, 55% of free device memory)",
            "offered_sweep_tflop_per_s": work / args.serve_seconds / 1e12 if args.serve_seconds else None}


def run_full_shapes(rgf):
    """The batching and serving workloads at their stated shapes.

    * uneven: 64 devices (N log-uniform 50..1000, b in {64, ..., 320}), 512
      energies each, one server run; energy points per second of wall time.
    * poisson_200: Poisson arrivals at 200 requests/s during a 5 s window
      (N log-uniform 20..2000, b uniform 96..288, 128..1024 energies, admission
      capped at min(150 GB, 55% of free memory)).  The offered work is about
      three orders of magnitude above one GPU, so the run is cut off 60 s
      after the first arrival: offered, admitted and completed requests are
      reported, and p50/p99 latency over every offered request, a request not
      done at the cut-off counting with its age then (a lower bound).  To keep
      device memory bounded, requests draw their device from a pool of 48
      devices drawn on the GPU from the same distribution (the server copies a
      request's blocks when it admits it, so requests may share inputs).
    * sustainable: the same request distribution at 0.1 request/s for 60 s,
      all requests run to completion: whether the queue stays bounded
      (completion of the last request within 60 s of its arrival)."""
    import numpy as np
    import torch

    from synth.devices import serving_trace
    from synth.gpu_devices import random_device_gpu, uneven_shapes

    out = {}
    shapes = uneven_shapes(64, 3, N_lo=50, N_hi=1000, b_choices=[64, 96, 128, 192, 256, 320])
    devs = [random_device_gpu(N, b, s, metal_frac=0.25, gap_offset=0.6) for N, b, s in shapes]
    E = np.linspace(-2.0, 2.0, 512)
    torch.cuda.synchronize()
    with rgf.Server(slots=148, class_step=32, tuning="default") as sv:
        t0 = time.perf_counter()
        tickets = [sv.submit(d, E, 1e-5) for d in devs]
        res = [sv.poll(t, timeout_us=3_600_000_000) for t in tickets]
        wall = time.perf_counter() - t0
        st = sv.stats()
    del devs
    torch.cuda.empty_cache()
    out["uneven_512"] = {"devices": 64, "energies_per_device": 512, "energy_points": 64 * 512, "seconds": wall,
                         "value": 64 * 512 / wall, "unit": "energy-points/s", "completed": int(sum(r is not None for r in res)),
                         "engines": st["engines"], "steps": st["steps"], "fp64_reseeds": st["fp64_reseeds"],
                         "flags_nonzero": int(sum(int(np.count_nonzero(r[2] & ~rgf.RGF_FLAG_REFINE))
                                                  for r in res if r is not None))}

    def serve(rate, window, cutoff, pool_n, seed):
        trace = serving_trace(seed, rate=rate, duration=window, N_lo=20, N_hi=2000, b_lo=96, b_hi=288,
                              nE_lo=128, nE_hi=1024)
        pool_tr = serving_trace(seed + 100, rate=1000.0, duration=pool_n / 1000.0 * 3, N_lo=20, N_hi=2000,
                                b_lo=96, b_hi=288, nE_lo=128, nE_hi=1024)[:pool_n]
        pool = [random_device_gpu(r["N"], r["b"], r["seed"], metal_frac=0.25, gap_offset=0.6) for r in pool_tr]
        rng = np.random.default_rng(seed)
        pick = rng.integers(0, len(pool), len(trace))
        torch.cuda.synchronize()
        lat, done_pts = [], 0
        with rgf.Server(slots=148, class_step=32, tuning="default") as sv:
            tickets = []
            t0 = time.perf_counter()
            for r, j in zip(trace, pick):
                delay = t0 + r["t"] - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                try:
                    tickets.append((sv.submit(pool[j], r["E"], r["eta"]), time.perf_counter(), r["n_E"], pool[j]))
                except rgf.RGFError:
                    tickets.append((None, time.perf_counter(), r["n_E"], pool[j]))
            pending = [t for t in tickets if t[0] is not None]
            while pending and time.perf_counter() - t0 < cutoff:
                nxt = []
                for t in pending:
                    res = sv.poll(t[0], timeout_us=0)
                    if res is None:
                        nxt.append(t)
                    else:
                        lat.append(res[3])
                        done_pts += t[2]
                pending = nxt
                if pending:
                    time.sleep(0.05)
            t_end = time.perf_counter()
            st = sv.stats()
            ages = [(t_end - t[1]) * 1e3 for t in tickets if t[0] is None] + [(t_end - t[1]) * 1e3 for t in pending]
        del pool
        torch.cuda.empty_cache()
        allv = sorted(lat + ages)
        pct = lambda q: allv[min(len(allv) - 1, int(round(q / 100 * (len(allv) - 1))))] if allv else None
        return {"rate_per_s": rate, "window_s": window, "cutoff_s": cutoff, "offered": len(trace),
                "admitted": int(st["submitted"] - st["rejected"]), "completed": len(lat),
                "not_done_at_cutoff": len(ages), "energy_points_done": done_pts,
                "energy_points_per_s": done_pts / (t_end - t0),
                "p50_ms_all_offered": pct(50), "p99_ms_all_offered": pct(99),
                "p50_ms_completed": float(np.median(lat)) if lat else None,
                "max_ms_completed": float(max(lat)) if lat else None,
                "peak_resident_bytes": st["peak_resident_bytes"], "device_pool": len(pool_tr)}

    out["poisson_200"] = serve(200.0, 5.0, 60.0, 48, 4)
    out["sustainable_0.1"] = serve(0.1, 60.0, 240.0, 8, 5)
    return out


def run_kpm(args, rgf):
    """Non-orthogonal KPM Fermi level of the 200-layer b = 128 junction
    (25,600 orbitals): power-iteration scale (100 steps), moments from
    random-phase vectors (one CTA each), E_F at half filling.  FP64 on the
    CUDA cores; the roofline is the FP64 pipe: 6 b x b block-vector products
    per layer, step and vector (H v: 3, forward substitution: 1, backward:
    2), 8 real flop per complex multiply-add."""
    import numpy as np
    import torch

    from synth import make_workload
    from synth.devices import random_phase_vectors

    dev, _, _ = make_workload("junction_N200_b128")
    N, b = dev.n_layers, dev.b
    R = random_phase_vectors(args.kpm_vectors, N * b, seed=21)
    x0 = random_phase_vectors(1, N * b, seed=22)[0]
    M = args.kpm_moments
    with rgf.KPM(dev) as k:
        t0 = time.perf_counter()
        alpha, beta = k.scale(x0, 100, 0.05)
        t_scale = time.perf_counter() - t0
        k.moments(R[:2], 4, alpha, beta)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mu = k.moments(R, M, alpha, beta)
        t_mom = time.perf_counter() - t0
        E_F = k.fermi_level(mu, alpha, beta, float(N * b))
    flops = 8.0 * 6 * b * b * N * args.kpm_vectors * (M - 1)
    return {"workload": "junction_N200_b128", "orbitals": N * b, "moments": M, "random_vectors": args.kpm_vectors,
            "alpha": alpha, "E_F": E_F, "scale_seconds": t_scale, "moments_seconds": t_mom,
            "fp64_tflops": flops / t_mom / 1e12,
            "note": "one CTA per random vector, whole recursion in one launch; FP64 pipe bound"}


def run_kpoints(args, rgf):
    """Transverse-periodic junction (R in {0, +1, -1}, 64 layers, b = 128)
    on an n x 1 Monkhorst-Pack mesh, 64 energies per k-point: Bloch sums,
    one server request per k-point and the mesh average, all on the GPU."""
    import numpy as np

    from synth.devices import monkhorst_pack, periodic_kdevice

    kd = periodic_kdevice(64, 128, 5)
    k, w = monkhorst_pack(args.kpoints)
    E = np.linspace(-1.5, 1.5, 64)
    with rgf.Server(slots=148, class_step=32, tuning="default") as sv:
        rgf.kpoint_transmission(sv, kd, k[:1], w[:1], E[:4], 1e-5)  # warm-up: engine creation
        t0 = time.perf_counter()
        T, Tk = rgf.kpoint_transmission(sv, kd, k, w, E, 1e-5, group=args.kpoints)
        dt = time.perf_counter() - t0
    return {"workload": "periodic_junction_N64_b128", "kpoints": int(len(k)), "energies": int(len(E)),
            "seconds": dt, "value": len(k) * len(E) / dt, "unit": "energy-k-points/s",
            "T_mean_range": [float(T.min()), float(T.max())]}


def run_ldos(args, rgf):
    """Layer-resolved DOS of the 200-layer b = 128 junction at n energies
    (mixed plan: forward sweep keeping every g_i, backward recursion)."""
    import numpy as np

    from synth import make_workload

    dev, E_all, eta = make_workload("junction_N200_b128")
    E = np.ascontiguousarray(E_all[: args.ldos_energies])
    with rgf.Plan(dev.n_layers, dev.b, precision=rgf.RGF_MIXED, eta=eta) as p:
        p.set_device(dev)
        p.ldos(E[:2])  # warm-up
        t0 = time.perf_counter()
        D = p.ldos(E)
        dt = time.perf_counter() - t0
    return {"workload": "junction_N200_b128", "energies": int(len(E)), "layers": dev.n_layers,
            "seconds": dt, "value": len(E) / dt, "unit": "energy-points/s (all layers)",
            "D_range": [float(D.min()), float(D.max())]}


def main():
    args = parse()
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import numpy as np
    import torch

    from paper_2609_37058_b300 import rgf
    from synth import make_workload

    torch.cuda.set_device(local)
    dev, E_all, eta = make_workload(WORKLOAD)
    n_E = len(E_all)
    W = args.wave
    prec = rgf.RGF_MIXED if args.precision == "mixed" else rgf.RGF_FP64
    stream = torch.cuda.Stream()
    plan = rgf.Plan(dev.n_layers, dev.b, precision=prec, eta=eta, energy_wave=W, cuda_stream=stream.cuda_stream)
    plan.set_device(dev)
    E_d = torch.tensor(E_all, dtype=torch.float64, device="cuda")
    T_d = torch.zeros(n_E, dtype=torch.float64, device="cuda")
    err_d = torch.zeros(n_E, dtype=torch.float64, device="cuda")
    flags_d = torch.zeros(n_E, dtype=torch.int32, device="cuda")

    from paper_2609_37058_b300.sharding import step_wave

    def wave(k):
        return step_wave(n_E, W, rank, world, k)

    def step(k):
        s, c = wave(k)
        rgf.rgf_transmission(plan.handle, E_d[s:s + c], T_d[s:s + c], err_d[s:s + c], flags_d[s:s + c])
        return c

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    clocks = ClockSampler(local)
    rgf.rgf_gemm_timing(True)
    launches0 = rgf.rgf_launch_count()
    phase0 = rgf.rgf_plan_phase_ms(plan.handle)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step_ms = []
    ev0.record(stream)
    done = 0
    for k in range(args.warmup, args.warmup + args.steps):
        a = torch.cuda.Event(enable_timing=True)
        b_ = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        done += step(k)
        b_.record(stream)
        step_ms.append((a, b_))
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks.stop()
    launches = rgf.rgf_launch_count() - launches0
    phase1 = rgf.rgf_plan_phase_ms(plan.handle)
    gemm_ms, gemm_n, gemm_flops = rgf.rgf_gemm_timing(False)
    elapsed = ev0.elapsed_time(ev1) / 1e3
    per_step = [a.elapsed_time(b_) for a, b_ in step_ms]
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([elapsed], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed = float(t.item())
        n = torch.tensor([done], device="cuda", dtype=torch.float64)
        dist.all_reduce(n)
        done_all = float(n.item())
    else:
        done_all = float(done)
    value = done_all / elapsed
    T_timed = T_d.cpu().numpy()
    fl = flags_d.cpu().numpy()
    ts, tc_ = wave(args.warmup)
    fl_t = fl[ts:ts + tc_]
    flag_counts = {"refine": int(np.sum((fl_t & rgf.RGF_FLAG_REFINE) != 0)),
                   "singular": int(np.sum((fl_t & rgf.RGF_FLAG_SINGULAR) != 0)),
                   "noconv": int(np.sum((fl_t & (rgf.RGF_FLAG_NOCONV_L | rgf.RGF_FLAG_NOCONV_R)) != 0)),
                   "max_err_estimate": float(err_d.cpu().numpy()[ts:ts + tc_].max())}

    if rank != 0:
        plan.close()
        return

    # ---------------------------------------------------------- end to end
    # The public call a user makes, from pinned host buffers (filled before
    # the timed region): upload the blocks and leads, then T(E) for one wave
    # of host energies into host arrays.
    pinned = []

    def pin(a, dtype=None):
        a = np.asarray(a, dtype=dtype)
        t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        pinned.append(t)
        return t.numpy()

    from synth.devices import Device, Lead

    lead_fields = ("H00", "S00", "H10", "S10", "Hc", "Sc")
    dev_h = Device(H_diag=pin(dev.H_diag), S_diag=pin(dev.S_diag), H_lower=pin(dev.H_lower),
                   S_lower=pin(dev.S_lower),
                   lead_L=Lead(*(pin(getattr(dev.lead_L, f)) for f in lead_fields)),
                   lead_R=Lead(*(pin(getattr(dev.lead_R, f)) for f in lead_fields)), name=dev.name)
    s, c = wave(args.warmup)
    E_h = pin(E_all[s:s + c], np.float64)
    T_h = pin(np.zeros(c), np.float64)
    err_h = pin(np.zeros(c), np.float64)
    fl_h = pin(np.zeros(c, dtype=np.int32))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan.set_device(dev_h)
    rgf.rgf_transmission(plan.handle, E_h, T_h, err_h, fl_h)
    e2e_s = time.perf_counter() - t0
    h2d = dev.nbytes() + sum(getattr(l, f).nbytes for l in (dev.lead_L, dev.lead_R)
                             for f in ("H00", "S00", "H10", "S10", "Hc", "Sc")) + E_h.nbytes
    d2h = T_h.nbytes + err_h.nbytes + fl_h.nbytes
    waves_done, reseeds = plan.stats
    plan.close()

    # ---------------------------------------------------------- FP64 GPU path
    # The same path in plain FP64 on the same GPU: one untimed warm-up wave,
    # then one wave of fp64_wave energies (the mixed step's first timed
    # energies) timed with CUDA events on the plan's stream, inputs resident.
    fp64 = None
    if not args.no_compare and prec == rgf.RGF_MIXED:
        Wf = args.fp64_wave
        s0f, _ = wave(args.warmup)
        with rgf.Plan(dev.n_layers, dev.b, precision=rgf.RGF_FP64, eta=eta, energy_wave=Wf,
                      cuda_stream=stream.cuda_stream) as pf:
            pf.set_device(dev)
            Ef = E_d[s0f:s0f + Wf]
            Tf = torch.zeros_like(Ef)
            rgf.rgf_transmission(pf.handle, E_d[:8], Tf[:8])  # warm-up
            torch.cuda.synchronize()
            fa, fb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            fa.record(stream)
            rgf.rgf_transmission(pf.handle, Ef, Tf)
            fb.record(stream)
            torch.cuda.synchronize()
            dtf = fa.elapsed_time(fb) / 1e3
        Tf = Tf.cpu().numpy()
        fp64 = {"value": Wf / dtf, "unit": "energy-points/s", "energies": Wf, "seconds": dtf,
                "timing": "one wave after a warm-up wave, CUDA events on the plan's stream",
                "max_abs_dT_vs_mixed": float(np.abs(Tf - T_timed[s0f:s0f + Wf]).max())}

    # ---------------------------------------------------------- CPU oracle
    s0, _ = wave(args.warmup)
    nb = args.cpu_energies
    T_cpu, cpu_s, threads, iters = oracle_sample(dev, E_all[s0:], eta, nb, info=True)
    dT = np.abs(T_cpu - T_timed[s0:s0 + nb])

    # ---------------------------------------------------------- method roofline
    # Throughput x the method's flop per energy (decimation iterations from the
    # oracle sample) against the measured FP64, TF32 and BF16 peaks.
    it_L = float(np.mean([i[0] for i in iters]))
    it_R = float(np.mean([i[1] for i in iters]))
    F = method_flop_per_energy(dev.n_layers, dev.b, it_L, it_R)
    pk = {}
    if not args.no_peaks:
        from paper_2609_37058_b300 import kernel_bench
        pk = kernel_bench.peaks(reps=3)
    mpeaks, _ = measured_peaks()

    def fractions(rate):
        tf = rate * F / 1e12
        d = {"method_tflops": tf}
        if pk:
            d["frac_of_fp64_peak"] = tf / pk["fp64_fma_tflops"]
            d["frac_of_tf32_peak"] = tf / pk["tf32_gemm_cublas_tflops"]
        d["frac_of_bf16_sustained"] = tf / float(mpeaks.get("bf16_tflops_sustained", 1400.0))
        return d

    method_roof = {"flop_per_energy": F, "decimation_iters": [it_L, it_R],
                   "count": "32b^3(N-1) + 8b^3 + 56b^3(iters_L + iters_R) + 32b^3 + 24b^3",
                   "mixed": fractions(value), "fp64_gpu": fractions(fp64["value"]) if fp64 else None,
                   "peaks_measured_here": pk or None}
    parity = None if args.no_golden else golden_parity(
        rgf, dict(precision=prec, eta=eta, energy_wave=W, cuda_stream=stream.cuda_stream), dev,
        args.parity_report)

    peaks, peak_src = measured_peaks()
    peak = float(peaks.get("bf16_tflops_sustained", 1400.0))
    roof = None
    if gemm_ms > 0:
        achieved = gemm_flops / (gemm_ms / 1e3) / 1e12
        traffic = None
        if GEMM_TRAFFIC is not None and GEMM_TRAFFIC[2] == tc_source_hash():
            traffic = GEMM_TRAFFIC[0] * (gemm_flops / gemm_n) / GEMM_TRAFFIC[1] if gemm_n else None
            # per launch, scaled from the captured launch by the flops ratio
        roof = {"bound": "tensor", "kernel": "k_oz_tc_p (persistent slice-product GEMM, tcgen05)", "achieved": achieved,
                "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                "peak_source": f"bf16_tflops_sustained of {peak_src}", "launches": gemm_n,
                "avg_launch_ms": gemm_ms / max(gemm_n, 1),
                "work": "BF16 flops of 21 slice-pair products, 2*M*N*K each (M=b, N=2b, K=2b)"}
    clk = clocks.summary()
    steps_sorted = sorted(per_step)
    p99 = steps_sorted[min(len(steps_sorted) - 1, int(round(0.99 * (len(steps_sorted) - 1))))]
    line = {
        "metric": METRIC, "value": value, "unit": "energy-points/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed * 1e3 / args.steps, "p50_ms": statistics.median(per_step),
        "p99_ms": p99, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16-slices/df32" if prec == rgf.RGF_MIXED else "f64",
        "data": "synthetic (seeded doped-junction Hamiltonian, Pt-Si:P-Pt-like)",
        "config": {"workload": WORKLOAD, "n_layers": dev.n_layers, "b": dev.b, "energies_per_step": W,
                   "eta": eta, "precision": args.precision, "parallelism": f"energy waves x{world}",
                   "l2": "inputs larger than L2 (2.1 GB of blocks, GBs of wave workspace)"},
        "gpu_launches": int(launches),
        "e2e": {"value": c / e2e_s, "unit": "energy-points/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "roofline": roof,
        "cpu_baseline": {"value": nb / cpu_s, "unit": "energy-points/s", "cores": threads, "kind": "oracle",
                         "sample": f"first {nb} energies of the first timed wave, numpy FP64 oracle"},
        "parity_sample": {"energies": nb, "max_abs_dT": float(dT.max()), "bar": 1e-6},
        "parity_stored_energies": parity,
        "method_roofline": method_roof,
        "fp64_gpu": fp64,
        "fp64_reseeds": reseeds,
        "phases_ms_per_step": {"lead_decimation_sigma_gamma": (phase1[0] - phase0[0]) / args.steps,
                               "layer_sweep_and_trace": (phase1[1] - phase0[1]) / args.steps},
        "flags_first_timed_wave": flag_counts,
        "clocks": clk,
    }
    if args.batch_energies > 0:
        line["batched"] = run_batched(args, rgf)
    if args.serve_seconds > 0:
        line["serving"] = run_serving(args, rgf)
    if args.kpoints > 0:
        line["kpoints"] = run_kpoints(args, rgf)
    if args.ldos_energies > 0:
        line["ldos"] = run_ldos(args, rgf)
    if args.kpm_moments > 0:
        line["kpm"] = run_kpm(args, rgf)
        if pk:
            line["kpm"]["frac_of_fp64_peak"] = line["kpm"]["fp64_tflops"] / max(pk["fp64_fma_tflops"],
                                                                                pk["fp64_dgemm_cublas_tflops"])
    if args.full_shapes:
        line["full_shapes"] = run_full_shapes(rgf)
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
