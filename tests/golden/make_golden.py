"""Write the FP64 oracle's T(E) for the named synthetic workloads.

Calls only ``oracle/`` and ``synth/``.  Output: one text file per workload,
``<name>.txt``, with columns index, E, T (repr precision).  The parity tests
compare the CUDA path against these rows; any change to the oracle's
arithmetic must regenerate them.

Usage: python tests/golden/make_golden.py [name ...]
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import rgf_oracle as o  # noqa: E402
from synth import make_workload  # noqa: E402

# name -> stride through the energy grid
PLAN = {"small_N64_b8": 1, "junction_N200_b128": 1, "doped_N500_b256": 16}


def write(name, stride):
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


if __name__ == "__main__":
    names = sys.argv[1:] or list(PLAN)
    for n in names:
        write(n, PLAN[n])
