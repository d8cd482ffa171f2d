"""FP64 CPU oracle for quantities derived from T(E).  TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import or run this module; the CUDA library shares no code
with it.

Landauer current, the paper's Eq. (1) in its linear-response form (the
transmission is the zero-bias T(E); only the electrode electrochemical
potentials move with the bias, Methods):

    I(V) = (2e/h) * integral dE [f(E, mu_L) - f(E, mu_R)] T(E),

with the readings mu_L = E_F + V/2 and mu_R = E_F - V/2 (the paper does not
split the bias), the Fermi-Dirac f(E, mu) = 1 / (1 + exp((E - mu)/kT)) (the
step with f = 1/2 at E = mu when kT = 0) and the trapezoidal rule on the
energy grid (the paper names no quadrature).  Energies in eV, current in A:
I = G0 * (integral in eV), G0 = 2 e^2 / h.

Layer-resolved density of states (the paper reports the spatially resolved
LDOS of its finite-bias runs; it gives no formula).  Reading: the Mulliken
partition of the device DOS in the nonorthogonal basis,

    D_i(E) = -(1/pi) Im Tr[(G S)_ii],  (G S)_ii = sum_j G_ij S_ji,

with G = (zS - H - Sigma_L (+) Sigma_R)^-1 the retarded device Green's
function (z = E + i eta), j running over the device layers only (the
overlap of the end layers with lead cells is not part of the device-region
partition); the D_i sum to -(1/pi) Im Tr[G S].  ``ldos`` is that definition
written out with a dense inverse.

Pins (``tests/test_oracle_observables.py``): unit transmission gives
I = G0 V (exactly at kT = 0 with the window edges on grid points, and to the
quadrature error at kT > 0); a linear T(E) at kT = 0 gives the exact
G0 V T(E_F); I(-V) = -I(V); the small-bias slope is G0 T(E_F).
"""
from __future__ import annotations

import numpy as np

from . import rgf_oracle

G0 = 7.748091729863649e-5  # 2 e^2 / h in siemens (CODATA 2018 e and h, exact)


def fermi(x, kT):
    x = np.asarray(x, dtype=np.float64)
    if kT > 0:
        return 0.5 * (1.0 - np.tanh(0.5 * x / kT))
    return np.where(x < 0, 1.0, np.where(x > 0, 0.0, 0.5))


def current(E, T, V, E_F, kT):
    """I(V) in ampere for every bias in V (eV units as above)."""
    E = np.asarray(E, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    out = []
    for v in np.atleast_1d(np.asarray(V, dtype=np.float64)):
        g = T * (fermi(E - (E_F + 0.5 * v), kT) - fermi(E - (E_F - 0.5 * v), kT))
        out.append(G0 * float(np.sum(0.5 * (E[1:] - E[:-1]) * (g[1:] + g[:-1]))))
    return np.array(out)


def _dense_S(dev):
    N, b = dev.n_layers, dev.b
    S = np.zeros((N * b, N * b), dtype=np.complex128)
    for i in range(N):
        S[i * b:(i + 1) * b, i * b:(i + 1) * b] = dev.S_diag[i]
    for i in range(1, N):
        S[i * b:(i + 1) * b, (i - 1) * b:i * b] = dev.S_lower[i - 1]
        S[(i - 1) * b:i * b, i * b:(i + 1) * b] = np.conj(dev.S_lower[i - 1].T)
    return S


def ldos(dev, energies, eta):
    """D[k, i] = -(1/pi) Im Tr[(G S)_ii] at energy k for every layer i."""
    N, b = dev.n_layers, dev.b
    S = _dense_S(dev)
    out = np.zeros((len(energies), N))
    for k, E in enumerate(energies):
        z = complex(E, eta)
        se = rgf_oracle.self_energies(dev, z)
        G = np.linalg.inv(rgf_oracle.assemble_dense(dev, z, se["sigma_L"], se["sigma_R"]))
        d = np.einsum("ij,ji->i", G, S)  # diagonal of G S
        out[k] = -(1.0 / np.pi) * d.reshape(N, b).sum(axis=1).imag
    return out
