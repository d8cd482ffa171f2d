"""Pins of the k-point oracle (no GPU): closed form of a chain stack, and the
exact identity between an M-point k mesh and a ring of M transverse cells."""
import cmath

import numpy as np
import pytest

from oracle import kpoints as ok
from oracle import rgf_oracle as o
from synth.devices import chain_stack, monkhorst_pack, periodic_kdevice


def chain_T(E, eta, eps, t, N):
    """Closed form of the uniform chain at finite eta: lambda root of
    t l^2 - (z - eps) l + t = 0 with |l| < 1, Gamma = -2 t Im l,
    G_{0,N-1} = l^(N-1) / (t (1/l - l)), T = Gamma^2 |G|^2."""
    z = complex(E, eta)
    d = cmath.sqrt((z - eps) ** 2 - 4 * t * t)
    l1, l2 = ((z - eps) + d) / (2 * t), ((z - eps) - d) / (2 * t)
    lam = l1 if abs(l1) < 1 else l2
    gam = -2 * t * lam.imag
    G = lam ** (N - 1) / (t * (1 / lam - lam))
    return gam * gam * abs(G) ** 2


@pytest.mark.parametrize("k", [0.0, 0.125, 0.3, 0.5])
def test_chain_stack_is_a_chain_at_the_shifted_energy(k):
    N, eps, t, ty, eta = 12, 0.1, 1.0, 0.25, 1e-4
    kd = chain_stack(N, eps, t, ty)
    E = np.array([-1.7, -0.6, 0.05, 0.9, 1.9])
    T = o.transmission(ok.device_at_k(kd, [k, 0.0]), E, eta)
    eps_k = eps + 2 * ty * np.cos(2 * np.pi * k)
    ref = np.array([chain_T(e, eta, eps_k, t, N) for e in E])
    assert np.allclose(T, ref, rtol=1e-10, atol=1e-14)


def test_bloch_sum_phases_and_hermiticity():
    kd = periodic_kdevice(4, 6, 5)
    k = [0.37, 0.0]
    Hk = ok.bloch_sum(kd.H_diag, kd.R, k)
    # On-site blocks are Hermitian at every k because X(-R) = X(R)^dagger.
    assert np.allclose(Hk, np.conj(np.swapaxes(Hk, -1, -2)), atol=1e-14)
    # k = 0 is the plain sum over R; k = 1 is the same as k = 0.
    assert np.allclose(ok.bloch_sum(kd.H_lower, kd.R, [0, 0]), kd.H_lower.sum(axis=0))
    assert np.allclose(ok.bloch_sum(kd.H_lower, kd.R, [1.0, 0]), kd.H_lower.sum(axis=0), atol=1e-13)


@pytest.mark.parametrize("M", [2, 3, 4])
def test_ring_of_M_cells_equals_sum_over_the_M_point_mesh(M):
    kd = periodic_kdevice(5, 4, 11, transverse=0.4)
    E = np.array([-1.1, -0.2, 0.45, 1.3])
    eta = 1e-5
    ks = [[m / M, 0.0] for m in range(M)]
    _, Tk = ok.transmission_kmesh(kd, ks, np.full(M, 1.0 / M), E, eta)
    T_ring = o.transmission(ok.ring_device(kd, M), E, eta)
    assert np.allclose(T_ring, Tk.sum(axis=0), rtol=1e-9, atol=1e-12)


def test_mesh_average_weights():
    kd = periodic_kdevice(3, 4, 2)
    k, w = monkhorst_pack(4)
    E = np.array([-0.5, 0.5])
    T, Tk = ok.transmission_kmesh(kd, k, w, E, 1e-5)
    assert np.allclose(T, Tk.mean(axis=0), rtol=1e-14)
    assert np.isclose(w.sum(), 1.0)
