"""Pins for the FP64 oracle, each independent of the oracle's own code.

* the uniform nearest-neighbour chain, whose surface Green's function,
  self-energy, broadening, end-to-end propagator and transmission have a
  closed form at any finite eta (written out here from the quadratic the
  surface Green's function satisfies);
* brute-force dense inversion of the whole device against the block
  recursion (left and right sweeps) on tiny random devices;
* the surface fixed-point residual, Hermiticity and positivity of Gamma;
* exact symmetries: H -> H + cS shifts T(E) to T(E - c); a unitary gauge
  on every layer leaves T unchanged; a cut coupling gives T = 0; mirror
  symmetry T_LR = T_RL as eta -> 0; 0 <= T <= number of orbitals.
"""
import cmath
import math

import numpy as np
import pytest

from oracle import rgf_oracle as o
from synth import Lead, chain_device, random_device
from synth.devices import Device


def chain_lambda(z, eps, t):
    """The root of t l^2 - (z - eps) l + t = 0 with |l| < 1."""
    d = cmath.sqrt((z - eps) ** 2 - 4 * t * t)
    l1 = ((z - eps) + d) / (2 * t)
    l2 = ((z - eps) - d) / (2 * t)
    return l1 if abs(l1) < 1 else l2


@pytest.mark.parametrize("eta", [1e-2, 1e-6])
@pytest.mark.parametrize("N", [1, 2, 5, 64])
def test_chain_closed_form(eta, N):
    eps, t = 0.0, 1.0
    dev = chain_device(max(N, 2))
    if N == 1:
        dev = Device(H_diag=dev.H_diag[:1], S_diag=dev.S_diag[:1], H_lower=dev.H_lower[:0],
                     S_lower=dev.S_lower[:0], lead_L=dev.lead_L, lead_R=dev.lead_R)
    # 40 points: E = 0 is left out on purpose.  There the chain is bipartite
    # and decimation starts from g = 1/(i eta), which loses ~eps/eta^2 of
    # accuracy (a property of the decimation, measured separately below).
    for E in np.linspace(-3.0, 3.0, 40):
        z = complex(E, eta)
        lam = chain_lambda(z, eps, t)
        se = o.self_energies(dev, z)
        assert se["converged"]
        assert abs(se["g_L"][0, 0] - lam / t) <= 1e-11 * abs(lam / t)
        assert abs(se["g_R"][0, 0] - lam / t) <= 1e-11 * abs(lam / t)
        assert abs(se["sigma_L"][0, 0] - t * lam) <= 1e-11 * abs(lam)
        gam = -2 * t * lam.imag
        assert abs(se["gamma_R"][0, 0] - gam) <= 1e-11 * max(abs(gam), 1e-300) + 1e-300
        G = lam ** (N - 1) / (t * (1 / lam - lam))
        T_exact = gam * gam * abs(G) ** 2
        G_o = o.rgf_G1N(dev, z, se["sigma_L"], se["sigma_R"])[0, 0]
        assert abs(abs(G_o) - abs(G)) <= 1e-10 * abs(G) + 1e-300
        T = o.transmission_one(dev, E, eta)
        assert abs(T - T_exact) <= 1e-10 * max(T_exact, 1e-300) + 1e-300


def test_decimation_band_centre_of_bipartite_chain():
    """At E = 0 exactly the chain is bipartite and the first decimation step
    divides by i*eta; the result is still the closed form to ~eps/eta^2."""
    dev = chain_device(4)
    for eta in (1e-2, 1e-3):
        z = complex(0.0, eta)
        lam = chain_lambda(z, 0.0, 1.0)
        a, alpha, beta, _, _ = o.lead_blocks(dev.lead_R, z, "R")
        g, it, ok = o.sancho_rubio(a, alpha, beta)
        assert ok
        assert abs(g[0, 0] - lam) <= 1e-15 / eta ** 2


def test_chain_integer_steps():
    """As eta -> 0 the perfect chain transmits exactly one channel inside the
    band |E| < 2|t| and nothing outside it."""
    dev = chain_device(16)
    E_in = np.array([-1.9, -1.0, 0.1, 0.5, 1.7])  # not E = 0 (see above)
    E_out = np.array([-2.5, 2.2, 3.0])
    T_in = o.transmission(dev, E_in, 1e-10)
    T_out = o.transmission(dev, E_out, 1e-10)
    assert np.all(np.abs(T_in - 1.0) < 1e-6)
    assert np.all(T_out < 1e-6)


def _tiny_device(N, b, seed):
    big = random_device(max(N, 2) + 2, b, seed, metal_frac=0.0)
    H_diag = big.H_diag[1:N + 1]
    S_diag = big.S_diag[1:N + 1]
    H_lower = big.H_lower[1:N]
    S_lower = big.S_lower[1:N]
    # Leads taken from the outer layers so that N = 1 works too.
    lead_L = Lead(H00=big.H_diag[0], S00=big.S_diag[0], H10=big.H_lower[0], S10=big.S_lower[0],
                  Hc=big.H_lower[0], Sc=big.S_lower[0])
    lead_R = Lead(H00=big.H_diag[-1], S00=big.S_diag[-1], H10=big.H_lower[-1],
                  S10=big.S_lower[-1], Hc=big.H_lower[-1], Sc=big.S_lower[-1])
    return Device(H_diag=H_diag, S_diag=S_diag, H_lower=H_lower, S_lower=S_lower,
                  lead_L=lead_L, lead_R=lead_R)


@pytest.mark.parametrize("N,b", [(1, 1), (1, 3), (2, 2), (3, 4), (6, 3), (5, 8)])
def test_rgf_equals_dense_inverse(N, b):
    dev = _tiny_device(N, b, seed=10 * N + b)
    for E in (-1.3, -0.2, 0.4, 1.1):
        z = complex(E, 1e-4)
        se = o.self_energies(dev, z)
        G_dense = o.dense_G1N(dev, z, se["sigma_L"], se["sigma_R"])
        G_left = o.rgf_G1N(dev, z, se["sigma_L"], se["sigma_R"])
        G_right = o.rgf_G1N_right_sweep(dev, z, se["sigma_L"], se["sigma_R"])
        nrm = np.linalg.norm(G_dense)
        assert np.linalg.norm(G_left - G_dense) <= 1e-11 * nrm
        assert np.linalg.norm(G_right - G_dense) <= 1e-11 * nrm
        # Brute force the inverse itself and read the corner block.
        Minv = np.linalg.inv(o.assemble_dense(dev, z, se["sigma_L"], se["sigma_R"]))
        assert np.linalg.norm(Minv[:b, (N - 1) * b:] - G_dense) <= 1e-11 * nrm
        T_rgf = o.transmission_one(dev, E, 1e-4)
        T_dense = o.transmission_one(dev, E, 1e-4, method="dense")
        assert abs(T_rgf - T_dense) <= 1e-11 * max(T_dense, 1e-12)


def test_dense_block_equals_full_inverse_entrywise():
    """The dense oracle path is itself the textbook definition: compare one
    block against an explicit inverse assembled entry by entry."""
    dev = _tiny_device(3, 2, seed=7)
    z = complex(0.3, 1e-3)
    se = o.self_energies(dev, z)
    b, N = 2, 3
    M = np.zeros((N * b, N * b), dtype=complex)
    for i in range(N):
        for r in range(b):
            for c in range(b):
                M[i * b + r, i * b + c] = z * dev.S_diag[i][r, c] - dev.H_diag[i][r, c]
    for i in range(1, N):
        for r in range(b):
            for c in range(b):
                low = z * dev.S_lower[i - 1][r, c] - dev.H_lower[i - 1][r, c]
                up = z * np.conj(dev.S_lower[i - 1][c, r]) - np.conj(dev.H_lower[i - 1][c, r])
                M[i * b + r, (i - 1) * b + c] = low
                M[(i - 1) * b + r, i * b + c] = up
    M[:b, :b] -= se["sigma_L"]
    M[-b:, -b:] -= se["sigma_R"]
    inv = np.linalg.inv(M)
    G = o.dense_G1N(dev, z, se["sigma_L"], se["sigma_R"])
    assert np.allclose(inv[:b, -b:], G, rtol=0, atol=1e-12 * np.abs(inv).max())


@pytest.mark.parametrize("eta", [1e-3, 1e-6])
def test_surface_gf_fixed_point_and_gamma(eta):
    dev = random_device(8, 6, seed=3)
    for E in np.linspace(-2.5, 2.5, 9):
        z = complex(E, eta)
        se = o.self_energies(dev, z)
        assert se["converged"]
        for side, g in (("L", se["g_L"]), ("R", se["g_R"])):
            lead = dev.lead_L if side == "L" else dev.lead_R
            a, alpha, beta, _, _ = o.lead_blocks(lead, z, side)
            resid = g - np.linalg.inv(a - alpha @ g @ beta)
            assert np.linalg.norm(resid) <= 1e-9 * np.linalg.norm(g)
            # Retarded branch: the anti-Hermitian part of g is negative.
            assert np.linalg.eigvalsh(1j * (g - g.conj().T)).min() >= -1e-9 * np.linalg.norm(g)
        for side, gam, g in (("L", se["gamma_L"], se["g_L"]), ("R", se["gamma_R"], se["g_R"])):
            lead = dev.lead_L if side == "L" else dev.lead_R
            _, _, _, c_low, c_up = o.lead_blocks(lead, z, side)
            nrm = np.linalg.norm(gam)
            assert np.linalg.norm(gam - gam.conj().T) <= 1e-14 * max(nrm, 1e-300)
            # Gamma = i(Sigma - Sigma^dag) is positive semidefinite when the
            # lead-device coupling is taken at real energy; eta in the
            # nonorthogonal coupling (z S_c) moves its spectrum by O(eta).
            two = lambda m: np.linalg.norm(m, 2)
            bound = 4 * eta * two(lead.Sc) * two(g) * max(two(c_low), two(c_up))
            assert np.linalg.eigvalsh(gam).min() >= -bound - 1e-12 * nrm


def test_gamma_psd_with_orthogonal_coupling():
    """With S_c = 0 the coupling is the same at z and at real E, and Gamma
    is exactly positive semidefinite."""
    dev = random_device(6, 5, seed=4)
    for lead in (dev.lead_L, dev.lead_R):
        lead.Sc = np.zeros_like(lead.Sc)
    for E in np.linspace(-2.5, 2.5, 7):
        se = o.self_energies(dev, complex(E, 1e-3))
        for gam in (se["gamma_L"], se["gamma_R"]):
            assert np.linalg.eigvalsh(gam).min() >= -1e-12 * max(np.linalg.norm(gam), 1e-300)


def _map_device(dev, f_diag, f_off):
    def lead(l):
        return Lead(H00=f_diag(l.H00, "H"), S00=f_diag(l.S00, "S"), H10=f_off(l.H10, "H"),
                    S10=f_off(l.S10, "S"), Hc=f_off(l.Hc, "H"), Sc=f_off(l.Sc, "S"))
    return Device(H_diag=np.array([f_diag(h, "H") for h in dev.H_diag]),
                  S_diag=dev.S_diag.copy(),
                  H_lower=np.array([f_off(h, "H") for h in dev.H_lower]),
                  S_lower=dev.S_lower.copy(), lead_L=lead(dev.lead_L), lead_R=lead(dev.lead_R))


def test_shift_by_overlap_shifts_energy():
    """z S - (H + c S) = (z - c) S - H, so T'(E) = T(E - c) exactly."""
    dev = random_device(6, 4, seed=5)
    c = 0.37
    shifted = Device(H_diag=dev.H_diag + c * dev.S_diag, S_diag=dev.S_diag,
                     H_lower=dev.H_lower + c * dev.S_lower, S_lower=dev.S_lower,
                     lead_L=Lead(H00=dev.lead_L.H00 + c * dev.lead_L.S00, S00=dev.lead_L.S00,
                                 H10=dev.lead_L.H10 + c * dev.lead_L.S10, S10=dev.lead_L.S10,
                                 Hc=dev.lead_L.Hc + c * dev.lead_L.Sc, Sc=dev.lead_L.Sc),
                     lead_R=Lead(H00=dev.lead_R.H00 + c * dev.lead_R.S00, S00=dev.lead_R.S00,
                                 H10=dev.lead_R.H10 + c * dev.lead_R.S10, S10=dev.lead_R.S10,
                                 Hc=dev.lead_R.Hc + c * dev.lead_R.Sc, Sc=dev.lead_R.Sc))
    E = np.linspace(-1.5, 1.5, 7)
    T0 = o.transmission(dev, E, 1e-4)
    T1 = o.transmission(shifted, E + c, 1e-4)
    assert np.allclose(T0, T1, rtol=1e-9, atol=1e-14)


def test_unitary_gauge_invariance():
    rng = np.random.default_rng(11)
    dev = random_device(5, 4, seed=6)
    N, b = dev.n_layers, dev.b
    U = [np.linalg.qr(rng.standard_normal((b, b)) + 1j * rng.standard_normal((b, b)))[0]
         for _ in range(N)]
    UL, UR = U[0], U[N - 1]
    tr = lambda X, P, Q: P @ X @ Q.conj().T
    g = Device(H_diag=np.array([tr(dev.H_diag[i], U[i], U[i]) for i in range(N)]),
               S_diag=np.array([tr(dev.S_diag[i], U[i], U[i]) for i in range(N)]),
               H_lower=np.array([tr(dev.H_lower[i - 1], U[i], U[i - 1]) for i in range(1, N)]),
               S_lower=np.array([tr(dev.S_lower[i - 1], U[i], U[i - 1]) for i in range(1, N)]),
               lead_L=Lead(H00=tr(dev.lead_L.H00, UL, UL), S00=tr(dev.lead_L.S00, UL, UL),
                           H10=tr(dev.lead_L.H10, UL, UL), S10=tr(dev.lead_L.S10, UL, UL),
                           Hc=tr(dev.lead_L.Hc, U[0], UL), Sc=tr(dev.lead_L.Sc, U[0], UL)),
               lead_R=Lead(H00=tr(dev.lead_R.H00, UR, UR), S00=tr(dev.lead_R.S00, UR, UR),
                           H10=tr(dev.lead_R.H10, UR, UR), S10=tr(dev.lead_R.S10, UR, UR),
                           Hc=tr(dev.lead_R.Hc, UR, U[N - 1]), Sc=tr(dev.lead_R.Sc, UR, U[N - 1])))
    E = np.linspace(-1.8, 1.8, 7)
    assert np.allclose(o.transmission(dev, E, 1e-4), o.transmission(g, E, 1e-4),
                       rtol=1e-9, atol=1e-14)


def test_cut_coupling_blocks_transport():
    dev = random_device(6, 3, seed=8)
    dev.H_lower[2] = 0.0
    dev.S_lower[2] = 0.0
    T = o.transmission(dev, np.linspace(-2, 2, 5), 1e-4)
    assert np.all(np.abs(T) < 1e-300 + 0.0) or np.all(np.abs(T) == 0.0)


def test_mirror_symmetry_small_eta():
    """Reversing the device (layer i -> N-1-i, lower <-> upper blocks, leads
    swapped) gives T_RL, which equals T_LR as eta -> 0."""
    dev = random_device(6, 3, seed=9)
    N = dev.n_layers
    dag = lambda m: np.conj(np.swapaxes(m, -1, -2))
    mir = Device(H_diag=dev.H_diag[::-1].copy(), S_diag=dev.S_diag[::-1].copy(),
                 H_lower=dag(dev.H_lower[::-1]).copy(), S_lower=dag(dev.S_lower[::-1]).copy(),
                 lead_L=Lead(H00=dev.lead_R.H00, S00=dev.lead_R.S00, H10=dag(dev.lead_R.H10),
                             S10=dag(dev.lead_R.S10), Hc=dag(dev.lead_R.Hc), Sc=dag(dev.lead_R.Sc)),
                 lead_R=Lead(H00=dev.lead_L.H00, S00=dev.lead_L.S00, H10=dag(dev.lead_L.H10),
                             S10=dag(dev.lead_L.S10), Hc=dag(dev.lead_L.Hc), Sc=dag(dev.lead_L.Sc)))
    E = np.linspace(-1.5, 1.5, 7)
    T = o.transmission(dev, E, 1e-10)
    Tm = o.transmission(mir, E, 1e-10)
    assert np.allclose(T, Tm, rtol=1e-6, atol=1e-9)


def test_transmission_bounds_and_real_trace():
    dev = random_device(10, 5, seed=12, metal_frac=0.3)
    E = np.linspace(-2.5, 2.5, 11)
    T, info = o.transmission(dev, E, 1e-6, return_info=True)
    assert np.all(T >= -1e-12)
    assert np.all(T <= dev.b + 1e-9)
    for i, t in zip(info, T):
        assert abs(i["trace_imag"]) <= 1e-9 * max(abs(t), 1e-9)


def test_decimation_stops_and_counts():
    dev = chain_device(4)
    z = complex(0.5, 1e-6)
    a, alpha, beta, _, _ = o.lead_blocks(dev.lead_R, z, "R")
    g, it, ok = o.sancho_rubio(a, alpha, beta)
    assert ok and 10 <= it <= 60
    g2, it2, ok2 = o.sancho_rubio(a, alpha, beta, max_iter=3)
    assert not ok2 and it2 == 3


def test_newton_refinement_drops_a_diverging_step():
    """Started from the advanced root of the uniform chain (|g alpha| > 1) the
    Newton step's doubling grows instead of converging: the step is dropped,
    g comes back unchanged and the refinement reports failure.  From the
    retarded root it holds and changes nothing."""
    z = complex(0.7, 1e-3)
    lam = chain_lambda(z, 0.0, 1.0)
    a = np.array([[z]], dtype=np.complex128)
    one = np.array([[1.0 + 0j]])
    g_adv = np.array([[1.0 / lam]])  # the other root of t l^2 - z l + t = 0: |g t| > 1
    assert abs(g_adv[0, 0]) > 1.0
    g, ok = o.newton_refine(a, one, one, g_adv.copy())
    assert not ok and np.array_equal(g, g_adv)
    g_ret = np.array([[lam]])
    g2, ok2 = o.newton_refine(a, one, one, g_ret.copy())
    assert ok2 and abs(g2[0, 0] - lam) <= 1e-14
