"""Pins of the current oracle (no GPU)."""
import numpy as np

from oracle import observables as ob


def test_G0_value():
    e, h = 1.602176634e-19, 6.62607015e-34  # exact SI values
    assert abs(ob.G0 - 2 * e * e / h) <= 1e-15 * ob.G0


def test_unit_transmission_zero_temperature_is_exact():
    # Spacing 2^-7 and biases that are multiples of 2^-6: the window edges
    # are exactly grid points, where the step takes its value 1/2.
    E = np.linspace(-1.0, 1.0, 257)
    for V in (0.125, 0.25, 0.5):
        I = ob.current(E, np.ones_like(E), [V], 0.0, 0.0)[0]
        assert abs(I - ob.G0 * V) <= 1e-14 * ob.G0 * V


def test_unit_transmission_finite_temperature():
    E = np.linspace(-2.0, 2.0, 8001)
    I = ob.current(E, np.ones_like(E), [0.1], 0.05, 0.025)[0]
    assert abs(I - ob.G0 * 0.1) <= 1e-6 * ob.G0 * 0.1


def test_linear_transmission_zero_temperature():
    E = np.linspace(-1.0, 1.0, 257)
    a, b, EF = 0.7, 0.3, 0.125
    for V in (0.125, 0.375):
        I = ob.current(E, a + b * E, [V], EF, 0.0)[0]
        assert abs(I - ob.G0 * V * (a + b * EF)) <= 1e-13 * ob.G0 * V


def test_antisymmetry_and_small_bias_slope():
    E = np.linspace(-1.0, 1.0, 2**14 + 1)  # spacing 2^-13
    T = 1.0 + 0.5 * np.sin(3 * E)
    I = ob.current(E, T, [0.02, -0.02], 0.0, 0.0)
    assert abs(I[0] + I[1]) <= 1e-15 * abs(I[0])
    V = 2.0**-8  # window edges +-2^-9 on grid points
    slope = ob.current(E, T, [V], 0.0, 0.0)[0] / V
    # I/V = G0 (T(E_F) + V^2 T''(E_F)/24 + quadrature error): T'' = 0 at 0.
    assert abs(slope - ob.G0 * 1.0) <= 1e-6 * ob.G0


def _chain_lambda(z, eps, t):
    import cmath
    d = cmath.sqrt((z - eps) ** 2 - 4 * t * t)
    l1, l2 = ((z - eps) + d) / (2 * t), ((z - eps) - d) / (2 * t)
    return l1 if abs(l1) < 1 else l2


def test_ldos_of_a_chain_window_is_the_bulk_site_dos():
    from synth import chain_device
    dev = chain_device(7)
    eta = 1e-6
    E = np.array([-1.5, -0.3, 0.8, 2.5])
    D = ob.ldos(dev, E, eta)
    for k, e in enumerate(E):
        lam = _chain_lambda(complex(e, eta), 0.0, 1.0)
        ref = -(1 / np.pi) * (1 / (1.0 * (1 / lam - lam))).imag
        assert np.allclose(D[k], ref, rtol=1e-9, atol=1e-12)


def test_ldos_mulliken_with_overlap_matches_k_integral():
    # Uniform chain with nearest-neighbour overlap s: the Mulliken site DOS
    # is the Brillouin-zone average of S(k) / (z S(k) - H(k)).
    from synth.devices import Device, Lead
    eps, t, s, N, eta = 0.1, 1.0, 0.15, 6, 2e-2
    one = np.ones((1, 1), complex)
    dev = Device(H_diag=np.full((N, 1, 1), eps, complex), S_diag=np.ones((N, 1, 1), complex),
                 H_lower=np.full((N - 1, 1, 1), t, complex), S_lower=np.full((N - 1, 1, 1), s, complex),
                 lead_L=Lead(eps * one, one, t * one, s * one, t * one, s * one),
                 lead_R=Lead(eps * one, one, t * one, s * one, t * one, s * one))
    E = np.array([-1.2, 0.0, 0.9])
    D = ob.ldos(dev, E, eta)
    k = (np.arange(200000) + 0.5) * (2 * np.pi / 200000)
    for i, e in enumerate(E):
        z = complex(e, eta)
        Sk, Hk = 1 + 2 * s * np.cos(k), eps + 2 * t * np.cos(k)
        ref = -(1 / np.pi) * np.mean(Sk / (z * Sk - Hk)).imag
        # Interior layers: every neighbour of the layer is in the device.  The
        # end layers also overlap lead cells, which the device-region
        # partition leaves out, so they differ.
        assert np.allclose(D[i, 1:-1], ref, rtol=1e-7), (e, D[i], ref)
        assert not np.isclose(D[i, 0], ref, rtol=1e-3)
