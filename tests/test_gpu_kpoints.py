"""Transverse k-point sampling on the GPU against the k-point oracle."""
import numpy as np
import pytest

from helpers import MIXED_ABS
from oracle import kpoints as ok
from synth.devices import chain_stack, monkhorst_pack, periodic_kdevice

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rgf():
    from paper_2609_37058_b300 import build, rgf as r
    build.build()
    return r


def test_bloch_sum_kernel(rgf):
    import torch
    kd = periodic_kdevice(5, 12, 4)
    for k in ([0.0, 0.0], [0.3125, 0.0], [-0.45, 0.0]):
        X = torch.as_tensor(kd.H_lower).cuda()
        Y = torch.empty(tuple(X.shape[1:]), dtype=torch.complex128, device="cuda")
        rgf.rgf_bloch_sum(kd.R, k, X, Y)
        ref = ok.bloch_sum(kd.H_lower, kd.R, k)
        assert np.abs(Y.cpu().numpy() - ref).max() <= 1e-14 * max(1.0, np.abs(ref).max())


def test_kmesh_mean_kernel(rgf):
    import torch
    rng = np.random.default_rng(0)
    Tk, w = rng.random((7, 33)), rng.random(7)
    out = torch.empty(33, dtype=torch.float64, device="cuda")
    rgf.rgf_kmesh_mean(torch.as_tensor(Tk).cuda(), torch.as_tensor(w).cuda(), out)
    assert np.abs(out.cpu().numpy() - w @ Tk).max() <= 1e-14


def test_kpoint_transmission_matches_oracle(rgf):
    kd = periodic_kdevice(6, 12, 9, transverse=0.4)
    k, w = monkhorst_pack(4)
    E = np.linspace(-1.2, 1.2, 9)
    eta = 1e-5
    with rgf.Server(slots=16, class_step=8) as sv:
        T, Tk = rgf.kpoint_transmission(sv, kd, k, w, E, eta, group=3)
    T_o, Tk_o = ok.transmission_kmesh(kd, k, w, E, eta)
    assert np.abs(Tk - Tk_o).max() <= MIXED_ABS
    assert np.abs(T - T_o).max() <= MIXED_ABS


def test_chain_stack_on_the_gpu(rgf):
    kd = chain_stack(20, 0.0, 1.0, 0.25)
    k, w = monkhorst_pack(5)
    E = np.array([-1.5, -0.4, 0.3, 1.1])
    with rgf.Server(slots=8, class_step=1) as sv:
        T, Tk = rgf.kpoint_transmission(sv, kd, k, w, E, 1e-4)
    T_o, Tk_o = ok.transmission_kmesh(kd, k, w, E, 1e-4)
    assert np.abs(Tk - Tk_o).max() <= MIXED_ABS and np.abs(T - T_o).max() <= MIXED_ABS
