"""Write the oracles' T(E) for the named synthetic workloads.

Calls only ``oracle/`` and ``synth/``.  Two kinds of file per workload:

* ``<name>.txt`` (default mode): the FP64 oracle (``oracle/rgf_oracle.py``),
  columns index, E, T (repr precision).
* ``<name>.ext.txt`` (``--ext``): the extended-precision oracle
  (``oracle/rgf_ext.c``, 64-bit significand), columns index, E, T, Im of the
  trace, left and right decimation iteration counts.

The parity tests compare the CUDA path against these rows; any change to an
oracle's arithmetic must regenerate its files.

Usage: python tests/golden/make_golden.py [--ext] [--threads K] [name ...]
"""
import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from synth import make_workload  # noqa: E402

# name -> stride through the energy grid
PLAN = {"small_N64_b8": 1, "junction_N200_b128": 1, "doped_N500_b256": 16}


def write_fp64(name, stride):
    from oracle import rgf_oracle as o
    dev, E, eta = make_workload(name)
    idx = np.arange(0, len(E), stride)
    t0 = time.time()
    T = o.transmission(dev, E[idx], eta)
    path = os.path.join(HERE, f"{name}.txt")
    with open(path, "w") as f:
        f.write(f"# FP64 oracle T(E) for workload {name} (eta = {eta!r}); energies idx::{stride} of "
                f"{len(E)}; written by tests/golden/make_golden.py in {time.time() - t0:.0f} s\n")
        f.write("# index E T\n")
        for i, e, t in zip(idx, E[idx], T):
            f.write(f"{int(i)} {float(e)!r} {float(t)!r}\n")
    print(path, len(idx), f"{time.time() - t0:.0f}s", flush=True)


def write_ext(name, stride, threads):
    if threads:
        os.environ["OMP_NUM_THREADS"] = str(threads)
    from oracle import rgf_ext as x
    dev, E, eta = make_workload(name)
    idx = np.arange(0, len(E), stride)
    t0 = time.time()
    T, info = x.transmission(dev, E[idx], eta, return_info=True)
    path = os.path.join(HERE, f"{name}.ext.txt")
    with open(path, "w") as f:
        f.write(f"# extended-precision (80-bit) oracle T(E) for workload {name} (eta = {eta!r}); "
                f"energies idx::{stride} of {len(E)}; written by tests/golden/make_golden.py --ext "
                f"in {time.time() - t0:.0f} s on {os.environ.get('OMP_NUM_THREADS', 'all')} threads\n")
        f.write("# index E T Im(trace) iters_L iters_R\n")
        for k, (i, e, t) in enumerate(zip(idx, E[idx], T)):
            f.write(f"{int(i)} {float(e)!r} {float(t)!r} {float(info['trace_imag'][k])!r} "
                    f"{int(info['iters'][k, 0])} {int(info['iters'][k, 1])}\n")
    print(path, len(idx), f"{time.time() - t0:.0f}s", flush=True)


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--ext", action="store_true")
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("names", nargs="*")
    a = ap.parse_args()
    for n in a.names or list(PLAN):
        if a.ext:
            write_ext(n, PLAN[n], a.threads)
        else:
            write_fp64(n, PLAN[n])
