"""Pins for the KPM oracle, each independent of its code.

* exact moments: with the scaled unit vectors sqrt(n) e_j as "random"
  vectors (their outer products average to I) the stochastic trace is the
  exact trace, and mu_n must equal sum_i T_n(lambda_i) over the
  generalized eigenvalues lambda_i = (eps_i - beta) / alpha from
  scipy.linalg.eigh(H, S) (a library generalized eigensolver);
* the integrated density of states counts those eigenvalues: at the centre
  of a spectral gap much wider than the kernel's resolution it is the
  integer number of eigenvalues below, and N(1) = mu_0 = the matrix size;
* the Fermi level for an electron count that fills whole levels lies in the
  gap between the last filled and the first empty eigenvalue;
* the stochastic estimator is unbiased: with random-phase vectors the
  moments of many vectors approach the exact ones within a few standard
  errors;
* the Jackson kernel's known values: g_0 = 1, g_{M-1} > 0 small, decreasing.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import kpm
from synth import random_device


def _setup(N, b, seed):
    dev = random_device(N, b, seed, metal_frac=0.25 if N >= 4 else 0.0, gap_offset=0.6)
    H, S = kpm.dense_blocks(dev)
    eps = scipy.linalg.eigh(H, S, eigvals_only=True)
    return dev, H, S, eps


@pytest.mark.parametrize("N,b,seed", [(3, 4, 1), (2, 7, 2), (5, 3, 3)])
def test_exact_moments_against_generalized_eigenvalues(N, b, seed):
    dev, H, S, eps = _setup(N, b, seed)
    alpha, beta = kpm.gershgorin_scale(H, S)
    assert np.all(np.abs((eps - beta) / alpha) < 1.0)
    lam = (eps - beta) / alpha
    n_mom = 40
    mu = kpm.moments(H, S, alpha, beta, np.sqrt(N * b) * np.eye(N * b), n_mom)
    exact = np.array([np.sum(np.cos(n * np.arccos(lam))) for n in range(n_mom)])
    assert np.allclose(mu, exact, rtol=0, atol=1e-10 * N * b)


def test_dense_blocks_are_hermitian_and_overlap_positive():
    dev, H, S, eps = _setup(4, 6, 7)
    assert np.allclose(H, H.conj().T) and np.allclose(S, S.conj().T)
    assert np.linalg.eigvalsh(S).min() > 0.5


def test_integrated_dos_counts_eigenvalues_in_gaps():
    dev, H, S, eps = _setup(3, 4, 1)
    alpha, beta = kpm.gershgorin_scale(H, S)
    n = N_b = len(eps)
    mu = kpm.moments(H, S, alpha, beta, np.sqrt(N_b) * np.eye(N_b), 3000)
    assert abs(kpm.states_below(mu, 1.0) - N_b) < 1e-9
    assert abs(kpm.states_below(mu, -1.0)) < 1e-9
    # the three widest gaps between consecutive eigenvalues
    gaps = np.argsort(np.diff(eps))[-3:]
    for k in gaps:
        mid = 0.5 * (eps[k] + eps[k + 1])
        width = eps[k + 1] - eps[k]
        assert width * 3000 / alpha > 20  # far wider than the kernel resolution
        x = (mid - beta) / alpha
        assert abs(kpm.states_below(mu, x) - (k + 1)) < 0.05, (k, kpm.states_below(mu, x))
    assert n == N_b


def test_fermi_level_in_the_selected_gap():
    dev, H, S, eps = _setup(3, 4, 1)
    alpha, beta = kpm.gershgorin_scale(H, S)
    mu = kpm.moments(H, S, alpha, beta, np.sqrt(len(eps)) * np.eye(len(eps)), 3000)
    k = int(np.argmax(np.diff(eps)))  # widest gap: k + 1 levels below it
    E_F = kpm.fermi_level(mu, alpha, beta, n_electrons=2.0 * (k + 1), spin=2.0)
    assert eps[k] < E_F < eps[k + 1]


def test_stochastic_estimator_is_unbiased():
    dev, H, S, eps = _setup(4, 6, 9)
    alpha, beta = kpm.gershgorin_scale(H, S)
    n_mom = 12
    exact = kpm.moments(H, S, alpha, beta, np.sqrt(len(eps)) * np.eye(len(eps)), n_mom)
    rng = np.random.default_rng(0)
    R = np.exp(2j * np.pi * rng.random((len(eps), 4000)))
    mu = kpm.moments(H, S, alpha, beta, R, n_mom)
    # per-vector estimates of Tr X have variance <= ||X||_F^2; 4000 vectors
    se = np.sqrt(len(eps)) / np.sqrt(4000)
    assert np.all(np.abs(mu - exact) < 5 * se)
    assert abs(mu[0] - len(eps)) < 1e-12  # |r_j| = 1 makes mu_0 exact


def test_jackson_kernel_values():
    g = kpm.jackson(64)
    assert abs(g[0] - 1.0) < 1e-15
    assert np.all(np.diff(g) < 0) and g[-1] > 0 and g[-1] < 1e-3


@pytest.mark.parametrize("N,b,seed", [(4, 64, 5), (6, 64, 6)])
def test_power_scale_covers_the_spectrum(N, b, seed):
    """At b = 64 the synthetic overlap is not diagonally dominant (no
    Gershgorin bound); 100 power steps on S^-1 H with a 5% margin still map
    every generalized eigenvalue of scipy.linalg.eigh(H, S) into [-1, 1],
    and not wastefully (alpha < 1.2 max |eps|)."""
    dev, H, S, eps = _setup(N, b, seed)
    with pytest.raises(ValueError):
        kpm.gershgorin_scale(H, S)
    x0 = np.exp(2j * np.pi * np.random.default_rng(seed).random(N * b))
    alpha, beta = kpm.power_scale(H, S, x0, 100, 0.05)
    assert beta == 0.0
    assert np.abs(eps).max() < alpha < 1.2 * np.abs(eps).max()
