"""FP64 CUDA path against the FP64 oracle, through the C ABI.

Bar: |dT| <= 1e-9 * max(T_oracle, 1e-6) per energy (relative 1e-9, with a
floor for transmissions below 1e-6 where a relative bar means nothing).
"""
import numpy as np
import pytest

from helpers import fp64_bar
from oracle import rgf_oracle as o
from synth import Lead, chain_device, make_workload, random_device
from synth.devices import Device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rgf():
    from paper_2609_37058_b300 import build, rgf as r
    build.build()
    return r


def run(rgf, dev, E, eta, **kw):
    with rgf.Plan(dev.n_layers, dev.b, eta=eta, **kw) as p:
        p.set_device(dev)
        return p.transmission(E)


def test_chain_closed_form_and_oracle(rgf):
    dev = chain_device(64)
    E = np.linspace(-3, 3, 256)
    T, err, flags = run(rgf, dev, E, 1e-6)
    T_o = o.transmission(dev, E, 1e-6)
    assert np.all(flags == 0)
    assert np.all(np.abs(T - T_o) <= fp64_bar(T_o))
    inside = np.abs(E) < 1.9
    assert np.all(np.abs(T[inside] - 1.0) < 1e-3)


def test_small_b8_all_energies(rgf):
    dev, E, eta = make_workload("small_N64_b8")
    T, err, flags = run(rgf, dev, E, eta)
    T_o = o.transmission(dev, E, eta)
    assert np.all(flags == 0)
    bad = np.abs(T - T_o) > fp64_bar(T_o)
    assert not bad.any(), (E[bad], T[bad], T_o[bad])


def _cut(N, b, seed):
    big = random_device(max(N, 2) + 2, b, seed)
    lead_L = Lead(big.H_diag[0], big.S_diag[0], big.H_lower[0], big.S_lower[0], big.H_lower[0],
                  big.S_lower[0])
    lead_R = Lead(big.H_diag[-1], big.S_diag[-1], big.H_lower[-1], big.S_lower[-1], big.H_lower[-1],
                  big.S_lower[-1])
    return Device(big.H_diag[1:N + 1].copy(), big.S_diag[1:N + 1].copy(), big.H_lower[1:N].copy(),
                  big.S_lower[1:N].copy(), lead_L, lead_R)


@pytest.mark.parametrize("N,b", [(1, 1), (1, 5), (2, 3), (3, 7), (5, 33), (4, 65), (3, 100)])
def test_ragged_shapes_against_dense(rgf, N, b):
    dev = _cut(N, b, seed=N * 100 + b)
    E = np.linspace(-1.7, 1.7, 9)
    T, err, flags = run(rgf, dev, E, 1e-4)
    T_o = o.transmission(dev, E, 1e-4, method="dense")
    assert np.all(np.abs(T - T_o) <= fp64_bar(T_o))


def test_junction_b128_sampled(rgf):
    dev, E, eta = make_workload("junction_N200_b128")
    idx = np.r_[0, 1, np.linspace(2, len(E) - 3, 6).astype(int), len(E) - 1]
    T, err, flags = run(rgf, dev, E[idx], eta)
    T_o = o.transmission(dev, E[idx], eta)
    assert np.all(flags == 0)
    d = np.abs(T - T_o)
    assert np.all(d <= fp64_bar(T_o)), (d, d / T_o)


def test_wave_split_and_determinism(rgf):
    dev = random_device(12, 24, seed=21, metal_frac=0.25, gap_offset=0.6)
    E = np.linspace(-2, 2, 37)
    T1, _, _ = run(rgf, dev, E, 1e-5)
    T2, _, _ = run(rgf, dev, E, 1e-5, energy_wave=5)   # ragged last wave of 2
    T3, _, _ = run(rgf, dev, E, 1e-5)
    assert np.array_equal(T1, T3)        # deterministic, bit for bit
    assert np.array_equal(T1, T2)        # waves are independent
    T_o = o.transmission(dev, E, 1e-5)
    assert np.all(np.abs(T1 - T_o) <= fp64_bar(T_o))


def test_device_pointers_and_async(rgf):
    import torch
    dev = random_device(10, 16, seed=5)
    E = np.linspace(-1.5, 1.5, 11)
    with rgf.Plan(dev.n_layers, dev.b, eta=1e-5) as p:
        p.set_device(dev)
        T_host, _, _ = p.transmission(E)
        Ed = torch.tensor(E, dtype=torch.float64, device="cuda")
        Td = torch.empty_like(Ed)
        rgf.rgf_transmission(p.handle, Ed, Td)
        assert np.array_equal(Td.cpu().numpy(), T_host)
        t1 = rgf.rgf_submit(p.handle, E)
        t2 = rgf.rgf_submit(p.handle, E[::-1].copy())
        T1 = np.empty_like(E)
        T2 = np.empty_like(E)
        assert rgf.rgf_poll(t1, T1, timeout_us=-1) == rgf.RGF_OK
        assert rgf.rgf_poll(t2, T2, timeout_us=-1) == rgf.RGF_OK
        assert np.array_equal(T1, T_host)
        assert np.array_equal(T2, T_host[::-1])


def test_nonconvergence_is_flagged(rgf):
    dev = random_device(4, 8, seed=2)
    E = np.array([-0.5, 0.5])
    T, err, flags = run(rgf, dev, E, 1e-6, dec_max_iter=2)
    assert np.all(flags & rgf.RGF_FLAG_NOCONV_L)
    assert np.all(flags & rgf.RGF_FLAG_NOCONV_R)
    # Same truncated decimation in the oracle gives the same T.
    T_o = o.transmission(dev, E, 1e-6, max_iter=2)
    assert np.all(np.abs(T - T_o) <= 1e-8 * np.maximum(np.abs(T_o), 1e-6))


def test_errors_on_bad_input(rgf):
    dev = random_device(4, 8, seed=2)
    with rgf.Plan(dev.n_layers, dev.b) as p:
        with pytest.raises(rgf.RGFError):
            p.transmission(np.array([0.0]))  # blocks not set yet
        H = dev.H_diag.copy()
        H[1][0, 1] += 1.0  # not Hermitian
        with pytest.raises(rgf.RGFError):
            rgf.rgf_set_device_blocks(p.handle, H, dev.S_diag, dev.H_lower, dev.S_lower)
        p.set_device(dev)
        T, _, _ = p.transmission(np.zeros(0))
        assert T.shape == (0,)


@pytest.mark.slow
def test_doped_b256_sampled(rgf):
    dev, E, eta = make_workload("doped_N500_b256")
    idx = np.array([0, 777, 1500, len(E) - 1])
    T, err, flags = run(rgf, dev, E[idx], eta)
    T_o = o.transmission(dev, E[idx], eta)
    assert np.all(flags == 0)
    d = np.abs(T - T_o)
    assert np.all(d <= fp64_bar(T_o)), (d, d / T_o)
