"""Autotuner of the server's per-class settings.

    python -m paper_2609_37058_b300.autotune --classes 64,96,128,192,256,320 \
        --out paper_2609_37058_b300/tuning_b300.json

For every block-size class the tuner times one synthetic junction (drawn on
the GPU, ``--layers`` layers, ``--energies`` energies) through the server
under candidate settings and keeps the fastest, by coordinate search:

1. the tensor-core tile width (64, 80 or 96 real output columns per CTA);
2. the Gauss-Jordan panel width of the FP32 seed inverse (16 or 32);
3. the number of energy slots (148, 74, then doubling from 296 while the
   rate improves, up to 1184; a candidate that does not fit in memory
   counts as the slowest); the smallest count within 3% of the best rate
   is kept, since slots cost device memory.

The figure of merit is energy points per second of wall time from
submission to result; each candidate runs on a fresh server after a short
warm-up request that creates the engine.  The table it writes is what
``rgf.Server(tuning="default")`` loads.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

TILES = (96, 80, 64)
PANELS = (32, 16)
SLOTS = (148, 74, 296)
MAX_SLOTS = 1184


def search(measure, bc: int, tol: float = 0.03):
    """Coordinate search over (tile_n, panel, slots); ``measure(bc, cfg)``
    returns energy points per second.  The slot count kept is the smallest
    whose rate is within ``tol`` of the best one measured (slots cost device
    memory).  Returns (best cfg, its rate, log)."""
    log = []

    def run(cfg):
        rate = float(measure(bc, dict(cfg)))
        log.append(dict(cfg, energy_points_per_s=rate))
        return rate

    cfg = {"tile_n": TILES[0], "panel": PANELS[0], "slots": SLOTS[0]}
    best = run(cfg)
    slot_rates = {cfg["slots"]: best}
    for key, values in (("tile_n", TILES), ("panel", PANELS), ("slots", SLOTS)):
        for v in values:
            if v == cfg[key]:
                continue
            trial = dict(cfg, **{key: v})
            rate = run(trial)
            if key == "slots":
                slot_rates[v] = rate
            if rate > best:
                best, cfg = rate, trial
        if key == "panel":
            slot_rates = {cfg["slots"]: best}
    # More slots keep paying while the launches are not yet full.
    s = max(SLOTS)
    while cfg["slots"] == s and s * 2 <= MAX_SLOTS:
        s *= 2
        trial = dict(cfg, slots=s)
        rate = run(trial)
        slot_rates[s] = rate
        if rate <= best:
            break
        best, cfg = rate, trial
    keep = min(n for n, r in slot_rates.items() if r >= (1.0 - tol) * best)
    if keep != cfg["slots"]:
        cfg = dict(cfg, slots=keep)
    return cfg, slot_rates[keep], log


def gpu_measure(layers: int, energies: int, eta: float = 1e-5):
    import torch

    from . import rgf
    from synth.gpu_devices import random_device_gpu

    def measure(bc, cfg):
        n_E = max(energies, 2 * cfg["slots"])
        dev = random_device_gpu(layers, bc, 1000 + bc, metal_frac=0.25, gap_offset=0.6)
        warm = random_device_gpu(3, bc, 2000 + bc)
        E = np.linspace(-2.0, 2.0, n_E)
        torch.cuda.synchronize()
        try:
            with rgf.Server(slots=cfg["slots"], class_step=32, tuning={bc: cfg}) as sv:
                t = sv.submit(warm, E[:4], eta)
                if sv.poll(t, timeout_us=600_000_000) is None:
                    raise RuntimeError("warm-up request did not finish")
                t0 = time.perf_counter()
                t = sv.submit(dev, E, eta)
                r = sv.poll(t, timeout_us=1_800_000_000)
                dt = time.perf_counter() - t0
        except rgf.RGFError as ex:
            if ex.status != rgf.RGF_E_OOM:
                raise
            return 0.0  # does not fit
        finally:
            del dev, warm
            torch.cuda.empty_cache()
        if r is None:
            raise RuntimeError("tuning request did not finish")
        return n_E / dt

    return measure


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--classes", default="64,96,128,160,192,224,256,288,320")
    ap.add_argument("--layers", type=int, default=96)
    ap.add_argument("--energies", type=int, default=296)
    ap.add_argument("--out", default=None, help="JSON file to write (default: print only)")
    a = ap.parse_args(argv)
    import torch

    measure = gpu_measure(a.layers, a.energies)
    out = {"device": torch.cuda.get_device_name(), "layers": a.layers, "energies": a.energies,
           "metric": "energy points per second, one request through the server", "classes": {}}
    for bc in (int(x) for x in a.classes.split(",")):
        cfg, rate, log = search(measure, bc)
        out["classes"][str(bc)] = dict(cfg, energy_points_per_s=rate, candidates=log)
        print(json.dumps({"class": bc, **cfg, "energy_points_per_s": rate}), flush=True)
    if a.out:
        with open(a.out, "w") as f:
            json.dump(out, f, indent=1)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
