"""The stored oracle values (tests/golden) without a GPU: the files are the
oracles' current output, on the grids the workloads define, and the FP64
oracle meets the FP64 bar against the 80-bit oracle at every stored energy.

The last point is what makes the FP64 oracle a usable reference at the
1e-9 relative level.  Without the Newton refinement of the lead surface
Green's functions it fails at 2 of 256 energies of the b = 8 grid (index
139: 5.7x the bar) and at about 15% of the b = 128 grid (up to ~1000x),
all from Sancho-Rubio's loss of digits (tests/test_oracle_ext.py pins
that).
"""
import os

import numpy as np
import pytest

from helpers import FP64_REL
from oracle import rgf_ext as x
from oracle import rgf_oracle as o
from synth import make_workload

HERE = os.path.dirname(os.path.abspath(__file__))
NAMES = ["small_N64_b8", "junction_N200_b128", "doped_N500_b256"]


def load(name):
    g = np.loadtxt(os.path.join(HERE, "golden", f"{name}.txt"))
    e = np.loadtxt(os.path.join(HERE, "golden", f"{name}.ext.txt"))
    return g, e


@pytest.mark.parametrize("name", NAMES)
def test_files_match_the_workload_grids(name):
    g, e = load(name)
    _, E, _ = make_workload(name)
    assert np.array_equal(g[:, 0], e[:, 0])
    idx = g[:, 0].astype(int)
    assert np.array_equal(g[:, 1], E[idx]) and np.array_equal(e[:, 1], E[idx])
    # the 80-bit trace is real to its own rounding; every decimation converged
    assert np.all(np.abs(e[:, 3]) <= 1e-12 * np.maximum(np.abs(e[:, 2]), 1e-6))
    assert np.all(e[:, 4] > 0) and np.all(e[:, 5] > 0)


@pytest.mark.parametrize("name", NAMES)
def test_fp64_oracle_meets_the_fp64_bar_against_the_80_bit_oracle(name):
    g, e = load(name)
    bar = FP64_REL * np.maximum(np.abs(e[:, 2]), 1e-6)
    ratio = np.abs(g[:, 2] - e[:, 2]) / bar
    assert ratio.max() <= 1.0, (int(g[np.argmax(ratio), 0]), ratio.max())


def test_b8_files_are_the_oracles_current_output():
    g, e = load("small_N64_b8")
    dev, E, eta = make_workload("small_N64_b8")
    assert np.allclose(o.transmission(dev, E, eta), g[:, 2], rtol=1e-10, atol=1e-300)
    assert np.allclose(x.transmission(dev, E, eta), e[:, 2], rtol=1e-15, atol=1e-300)


def test_b128_files_are_the_oracles_current_output():
    g, e = load("junction_N200_b128")
    dev, E, eta = make_workload("junction_N200_b128")
    k = [0, 676]
    assert np.allclose(o.transmission(dev, E[k], eta), g[k, 2], rtol=1e-9, atol=0)
    assert np.allclose(x.transmission(dev, E[[676]], eta), e[[676], 2], rtol=1e-15, atol=0)
