"""Non-orthogonal KPM Fermi level on the GPU (rgf_kpm.h) against the KPM
oracle, through the C ABI, on the same seeded random vectors.

Bars: moments |d mu_n| <= 1e-10 mu_0 (FP64 recursion against FP64 dense
solves; mu_0 = N b for unit-modulus vectors); power-iteration scale to
1e-10 relative, and it covers every generalized eigenvalue of
scipy.linalg.eigh(H, S) within 20%; Fermi level from identical moments to 1e-12 eV and from each
side's own moments to 1e-9 eV.  With the scaled unit vectors as random
vectors the GPU moments equal the exact traces over the generalized
eigenvalues of scipy.linalg.eigh(H, S).
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import kpm as okpm
from synth import random_device
from synth.devices import random_phase_vectors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rgf():
    from paper_2609_37058_b300 import build, rgf as r
    build.build()
    return r


@pytest.mark.parametrize("N,b,n_rand,n_mom", [(1, 5, 3, 20), (2, 3, 4, 33), (5, 7, 6, 64), (4, 33, 5, 50),
                                              (3, 130, 2, 40)])
def test_moments_and_fermi_level_against_oracle(rgf, N, b, n_rand, n_mom):
    dev = random_device(max(N, 2), b, 40 + N * b, metal_frac=0.25, gap_offset=0.6)
    if N == 1:
        from synth.devices import Device
        dev = Device(dev.H_diag[:1], dev.S_diag[:1], dev.H_lower[:0], dev.S_lower[:0], dev.lead_L, dev.lead_R)
    H, S = okpm.dense_blocks(dev)
    R = random_phase_vectors(n_rand, N * b, seed=N * 1000 + b)
    x0 = random_phase_vectors(1, N * b, seed=3)[0]
    eps = scipy.linalg.eigh(H, S, eigvals_only=True)
    with rgf.KPM(dev) as k:
        alpha, beta = k.scale(x0, 100, 0.05)
        a_o, b_o = okpm.power_scale(H, S, x0, 100, 0.05)
        assert abs(alpha - a_o) <= 1e-10 * a_o and beta == b_o == 0.0
        assert np.abs(eps).max() <= alpha <= 1.2 * np.abs(eps).max()
        mu = k.moments(R, n_mom, alpha, beta)
        mu_o = okpm.moments(H, S, alpha, beta, R.T, n_mom)
        assert np.abs(mu - mu_o).max() <= 1e-10 * mu_o[0], np.abs(mu - mu_o).max()
        n_el = float(N * b)  # half filling, spin 2
        E_same = k.fermi_level(mu_o, alpha, beta, n_el)
        E_o = okpm.fermi_level(mu_o, alpha, beta, n_el)
        assert abs(E_same - E_o) <= 1e-12
        assert abs(k.fermi_level(mu, alpha, beta, n_el) - E_o) <= 1e-9


def test_exact_trace_moments_against_generalized_eigenvalues(rgf):
    dev = random_device(6, 9, 77, metal_frac=0.25, gap_offset=0.6)
    H, S = okpm.dense_blocks(dev)
    n = H.shape[0]
    eps = scipy.linalg.eigh(H, S, eigvals_only=True)
    with rgf.KPM(dev) as k:
        alpha, beta = k.scale(random_phase_vectors(1, n, seed=4)[0], 100, 0.05)
        mu = k.moments(np.sqrt(n) * np.eye(n), 48, alpha, beta)
    lam = (eps - beta) / alpha
    exact = np.array([np.sum(np.cos(m * np.arccos(lam))) for m in range(48)])
    assert np.abs(mu - exact).max() <= 1e-10 * n


def test_junction_sized_moments(rgf):
    """A 24-layer b = 64 junction (1536 orbitals), 16 vectors, 96 moments."""
    dev = random_device(24, 64, 5, metal_frac=0.25, gap_offset=0.6)
    H, S = okpm.dense_blocks(dev)
    R = random_phase_vectors(16, 24 * 64, seed=11)
    with rgf.KPM(dev) as k:
        alpha, beta = k.scale(random_phase_vectors(1, 24 * 64, seed=12)[0], 100, 0.05)
        mu = k.moments(R, 96, alpha, beta)
        E_F = k.fermi_level(mu, alpha, beta, 1536.0)
    mu_o = okpm.moments(H, S, alpha, beta, R.T, 96)
    assert np.abs(mu - mu_o).max() <= 1e-10 * mu_o[0]
    assert abs(E_F - okpm.fermi_level(mu_o, alpha, beta, 1536.0)) <= 1e-9


def test_invalid_arguments(rgf):
    import ctypes
    L = rgf.lib()
    h = ctypes.c_void_p()
    assert L.rgf_kpm_create(ctypes.byref(h), 0, 4, None, None, None, None, 0, None) == rgf.RGF_E_INVALID
    dev = random_device(3, 4, 1)
    with rgf.KPM(dev) as k:
        with pytest.raises(ValueError):
            k.moments(np.ones((2, 5), complex), 10, 1.0, 0.0)  # wrong vector length (caught in the binding)
        st = L.rgf_kpm_moments(k.handle, 0.0, 0.0, 1, None, 10, None)
        assert st == rgf.RGF_E_INVALID
        # a scale that leaves the spectrum outside [-1, 1] is refused
        R = random_phase_vectors(2, 12, seed=1)
        with pytest.raises(rgf.RGFError):
            k.moments(R, 200, 0.05, 0.0)
