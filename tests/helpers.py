"""Test-side helpers: the tolerance bars.

The FP64 bar is relative 1e-9 with a floor at T = 1e-6 (for T below 1e-6 a
relative bar means nothing); the mixed bar is 1e-6 absolute.  Both are
applied as they are: the lead surface Green's functions are refined by
Newton steps in the oracles and in the CUDA paths, which removes the loss of
digits of Sancho-Rubio decimation that had put the FP64 oracle itself
outside the FP64 bar at some energies (tests/test_oracle_ext.py,
tests/test_golden.py).
"""
import numpy as np

FP64_REL = 1e-9
MIXED_ABS = 1e-6


def fp64_bar(T_ref):
    return FP64_REL * np.maximum(np.abs(T_ref), 1e-6)
