"""Landauer current on the GPU against the current oracle."""
import numpy as np
import pytest

from oracle import observables as ob
from oracle import rgf_oracle as o
from synth import random_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rgf():
    from paper_2609_37058_b300 import build, rgf as r
    build.build()
    return r


def gpu_current(rgf, E, T, V, E_F, kT):
    import torch
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    I = torch.empty(len(V), dtype=torch.float64, device="cuda")
    rgf.rgf_current(t(E), t(T), t(V), E_F, kT, I)
    return I.cpu().numpy()


@pytest.mark.parametrize("kT", [0.0, 0.0257])
def test_current_kernel_matches_oracle(rgf, kT):
    rng = np.random.default_rng(3)
    E = np.linspace(-1.0, 1.0, 1025)
    T = rng.random(E.shape[0]) * 3
    V = np.array([-0.3, -0.1, 0.0, 0.05, 0.1, 0.2, 0.4])
    I = gpu_current(rgf, E, T, V, 0.03, kT)
    I_o = ob.current(E, T, V, 0.03, kT)
    assert np.allclose(I, I_o, rtol=1e-12, atol=1e-20)


def test_current_from_the_mixed_path(rgf):
    # T(E) from the mixed plan, then the current on the GPU, against the
    # oracle's T and current: |dI| <= G0 * integral |dT| dE <= G0 * 1e-6 * V.
    dev = random_device(12, 16, 4, metal_frac=0.25, gap_offset=0.6)
    E = np.linspace(-0.75, 0.75, 97)
    eta = 1e-5
    with rgf.Plan(dev.n_layers, dev.b, precision=rgf.RGF_MIXED, eta=eta) as p:
        p.set_device(dev)
        T, _, _ = p.transmission(E)
    T_o = o.transmission(dev, E, eta)
    V = np.array([0.1, 0.25, 0.5])
    I = gpu_current(rgf, E, T, V, 0.0, 0.01)
    I_o = ob.current(E, T_o, V, 0.0, 0.01)
    assert np.all(np.abs(I - I_o) <= ob.G0 * 1e-6 * (V + 0.1))


def test_ldos_matches_oracle(rgf):
    dev = random_device(7, 12, 8, metal_frac=0.3, gap_offset=0.6)
    E = np.linspace(-1.2, 1.2, 11)
    eta = 1e-4
    with rgf.Plan(dev.n_layers, dev.b, precision=rgf.RGF_MIXED, eta=eta) as p:
        p.set_device(dev)
        D = p.ldos(E)
    D_o = ob.ldos(dev, E, eta)
    assert np.all(np.abs(D - D_o) <= 1e-6 * np.maximum(1.0, np.abs(D_o))), np.abs(D - D_o).max()


def test_ldos_of_a_chain_window(rgf):
    from synth import chain_device
    dev = chain_device(9)
    E = np.array([-1.5, -0.3, 0.8, 1.7])
    with rgf.Plan(dev.n_layers, dev.b, precision=rgf.RGF_MIXED, eta=1e-6) as p:
        p.set_device(dev)
        D = p.ldos(E)
    assert np.abs(D - ob.ldos(dev, E, 1e-6)).max() <= 1e-6


def test_ldos_needs_a_mixed_plan(rgf):
    dev = random_device(3, 4, 1)
    with rgf.Plan(dev.n_layers, dev.b, precision=rgf.RGF_FP64, eta=1e-5) as p:
        p.set_device(dev)
        with pytest.raises(rgf.RGFError) as ex:
            p.ldos(np.array([0.1]))
        assert ex.value.status == rgf.RGF_E_STATE
