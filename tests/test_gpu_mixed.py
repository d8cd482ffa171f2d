"""Mixed-precision CUDA path against the FP64 oracle through the C ABI.

Bar: |dT| <= 1e-6 absolute per energy.
"""
import os

import numpy as np
import pytest

from helpers import MIXED_ABS
from oracle import rgf_oracle as o
from synth import Lead, chain_device, make_workload, random_device
from synth.devices import Device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rgf():
    from paper_2609_37058_b300 import build, rgf as r
    build.build()
    return r


def run(rgf, dev, E, eta, core=None, **kw):
    if core is None:
        core = int(os.environ.get("RGF_TEST_CORE", "0"))
    os.environ["RGF_OZ_CORE"] = str(core)
    try:
        with rgf.Plan(dev.n_layers, dev.b, precision=rgf.RGF_MIXED, eta=eta, **kw) as p:
            p.set_device(dev)
            return p.transmission(E)
    finally:
        os.environ.pop("RGF_OZ_CORE", None)


@pytest.mark.parametrize("core", [0, 1], ids=["tc", "mma"])
def test_chain(rgf, core):
    dev = chain_device(64)
    E = np.linspace(-3, 3, 256)
    T, err, flags = run(rgf, dev, E, 1e-6, core=core)
    T_o = o.transmission(dev, E, 1e-6)
    assert np.all((flags & ~rgf.RGF_FLAG_REFINE) == 0)
    assert np.abs(T - T_o).max() <= MIXED_ABS


@pytest.mark.parametrize("core", [0, 1], ids=["tc", "mma"])
def test_small_b8(rgf, core):
    dev, E, eta = make_workload("small_N64_b8")
    T, err, flags = run(rgf, dev, E, eta, core=core)
    T_o = o.transmission(dev, E, eta)
    # RGF_FLAG_REFINE only reports an FP64 reseed of an ill-conditioned block.
    assert np.all((flags & ~rgf.RGF_FLAG_REFINE) == 0)
    assert np.abs(T - T_o).max() <= MIXED_ABS


def _cut(N, b, seed):
    big = random_device(max(N, 2) + 2, b, seed, metal_frac=0.25, gap_offset=0.6)
    lead_L = Lead(big.H_diag[0], big.S_diag[0], big.H_lower[0], big.S_lower[0], big.H_lower[0], big.S_lower[0])
    lead_R = Lead(big.H_diag[-1], big.S_diag[-1], big.H_lower[-1], big.S_lower[-1], big.H_lower[-1],
                  big.S_lower[-1])
    return Device(big.H_diag[1:N + 1].copy(), big.S_diag[1:N + 1].copy(), big.H_lower[1:N].copy(),
                  big.S_lower[1:N].copy(), lead_L, lead_R)


@pytest.mark.parametrize("N,b", [(1, 1), (1, 5), (2, 3), (3, 7), (5, 33), (4, 65), (3, 100), (6, 130)])
def test_ragged_shapes(rgf, N, b):
    dev = _cut(N, b, seed=N * 100 + b)
    E = np.linspace(-1.7, 1.7, 9)
    T, err, flags = run(rgf, dev, E, 1e-4)
    T_o = o.transmission(dev, E, 1e-4, method="dense")
    assert np.all((flags & ~rgf.RGF_FLAG_REFINE) == 0)
    assert np.abs(T - T_o).max() <= MIXED_ABS


def test_junction_b128_sampled(rgf):
    dev, E, eta = make_workload("junction_N200_b128")
    idx = np.r_[0, 1, np.linspace(2, len(E) - 3, 6).astype(int), len(E) - 1]
    T, err, flags = run(rgf, dev, E[idx], eta)
    T_o = o.transmission(dev, E[idx], eta)
    assert np.all((flags & ~rgf.RGF_FLAG_REFINE) == 0)
    d = np.abs(T - T_o)
    assert d.max() <= MIXED_ABS, d


def test_wave_split_and_determinism(rgf):
    dev = random_device(12, 24, seed=21, metal_frac=0.25, gap_offset=0.6)
    E = np.linspace(-2, 2, 37)
    T1, _, _ = run(rgf, dev, E, 1e-5)
    T2, _, _ = run(rgf, dev, E, 1e-5, energy_wave=5)
    T3, _, _ = run(rgf, dev, E, 1e-5)
    assert np.array_equal(T1, T3)
    assert np.array_equal(T1, T2)
    T_o = o.transmission(dev, E, 1e-5)
    assert np.abs(T1 - T_o).max() <= MIXED_ABS


@pytest.mark.slow
def test_doped_b256_sampled(rgf):
    dev, E, eta = make_workload("doped_N500_b256")
    idx = np.array([0, 777, 1500, len(E) - 1])
    T, err, flags = run(rgf, dev, E[idx], eta)
    T_o = o.transmission(dev, E[idx], eta)
    assert np.all((flags & ~rgf.RGF_FLAG_REFINE) == 0)
    d = np.abs(T - T_o)
    assert d.max() <= MIXED_ABS, d
