"""The block sizes of the uneven-device and serving workloads, against the
FP64 oracle through the C ABI.

* b = 288 and b = 320 (the largest block sizes the batched and serving
  workloads draw) through the single-device mixed plan and through the
  server, N = 8 layers, 8 energies each;
* a batch shaped like the uneven-device workload (every block size of
  {64, 96, 128, 192, 256, 320}, uneven lengths, one server run), every
  request checked.

Bar: |dT| <= 1e-6 absolute (the mixed path's), flags other than an FP64
reseed must be clear.
"""
import numpy as np
import pytest

from helpers import MIXED_ABS
from oracle import rgf_oracle as o
from synth import random_device
from synth.devices import energy_grid

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rgf():
    from paper_2609_37058_b300 import build, rgf as r
    build.build()
    return r


def _check(rgf, dev, E, eta, T, flags):
    T_o = o.transmission(dev, E, eta)
    assert np.all((flags & ~rgf.RGF_FLAG_REFINE) == 0), flags
    d = np.abs(T - T_o)
    assert d.max() <= MIXED_ABS, (dev.b, d.max(), E[np.argmax(d)])


@pytest.mark.parametrize("b", [288, 320])
def test_large_blocks_single_plan(rgf, b):
    dev = random_device(8, b, 700 + b, metal_frac=0.25, gap_offset=0.6)
    E = energy_grid(-1.4, 1.3, 8)
    with rgf.Plan(dev.n_layers, dev.b, precision=rgf.RGF_MIXED, eta=1e-5) as p:
        p.set_device(dev)
        T, err, flags = p.transmission(E)
    _check(rgf, dev, E, 1e-5, T, flags)


def test_large_blocks_server(rgf):
    jobs = [(random_device(8, b, 800 + b, metal_frac=0.25, gap_offset=0.6), energy_grid(-1.2, 1.5, 8), 1e-5)
            for b in (288, 320)]
    with rgf.Server(slots=16, class_step=32, tuning="default") as sv:
        tickets = [sv.submit(d, E, eta) for d, E, eta in jobs]
        res = [sv.poll(t, timeout_us=300_000_000) for t in tickets]
    assert all(r is not None for r in res)
    for (dev, E, eta), (T, err, flags, lat) in zip(jobs, res):
        _check(rgf, dev, E, eta, T, flags)


def test_uneven_batch_every_block_size(rgf):
    """One device per block size of the uneven-device workload, lengths 6 to
    13 (uneven), 8 energies each (eta = 1e-5 as that workload), all in one
    server run with the tuned per-class settings."""
    bs = [64, 96, 128, 192, 256, 320]
    Ns = [13, 6, 11, 9, 7, 8]
    jobs = [(random_device(N, b, 900 + b, metal_frac=0.25, gap_offset=0.6), energy_grid(-2.0, 2.0, 8), 1e-5)
            for N, b in zip(Ns, bs)]
    with rgf.Server(slots=148, class_step=32, tuning="default") as sv:
        tickets = [sv.submit(d, E, eta) for d, E, eta in jobs]
        res = [sv.poll(t, timeout_us=300_000_000) for t in tickets]
        st = sv.stats()
    assert all(r is not None for r in res)
    assert st["engines"] == len(bs)
    for (dev, E, eta), (T, err, flags, lat) in zip(jobs, res):
        _check(rgf, dev, E, eta, T, flags)
