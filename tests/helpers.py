"""Test-side helpers: tolerance bars and exact input transformations.

The FP64 bar is relative 1e-9 with a floor at T = 1e-6.  At a few energies
the FP64 problem itself is worse conditioned than that: the lead
broadening Gamma = i(Sigma - Sigma^dag) is a small difference of O(1)
self-energies when a lead is nearly closed, and decimation near a lead band
edge loses digits.  There the FP64 oracle's own rounding error exceeds
1e-9 (an 80-bit re-evaluation of the 64-layer b = 8 device shows the FP64
oracle off by 1.2e-8 relative at E = 0.2706).  ``fp64_uncertainty``
measures that rounding sensitivity without a second implementation: it
re-runs the oracle on the same device in random block-unitary gauges (an
exact symmetry of T) and takes the spread.  The bar used by the FP64
parity tests is max(1e-9 * max(T, 1e-6), 4 * spread).
"""
import numpy as np

from oracle import rgf_oracle as o
from synth.devices import Device, Lead

FP64_REL = 1e-9
MIXED_ABS = 1e-6


def gauge_transform(dev, rng):
    """Apply a random unitary U_i on every layer (leads take U_0 and U_{N-1})."""
    N, b = dev.n_layers, dev.b
    U = [np.linalg.qr(rng.standard_normal((b, b)) + 1j * rng.standard_normal((b, b)))[0]
         for _ in range(N)]
    UL, UR = U[0], U[-1]
    tr = lambda X, P, Q: P @ X @ Q.conj().T
    lead = lambda l, Ua, Uc: Lead(tr(l.H00, Ua, Ua), tr(l.S00, Ua, Ua), tr(l.H10, Ua, Ua),
                                  tr(l.S10, Ua, Ua), Uc[0](l.Hc), Uc[0](l.Sc))
    return Device(
        H_diag=np.array([tr(dev.H_diag[i], U[i], U[i]) for i in range(N)]),
        S_diag=np.array([tr(dev.S_diag[i], U[i], U[i]) for i in range(N)]),
        H_lower=np.array([tr(dev.H_lower[i - 1], U[i], U[i - 1]) for i in range(1, N)]).reshape(-1, b, b),
        S_lower=np.array([tr(dev.S_lower[i - 1], U[i], U[i - 1]) for i in range(1, N)]).reshape(-1, b, b),
        lead_L=lead(dev.lead_L, UL, (lambda X: tr(X, U[0], UL),)),
        lead_R=lead(dev.lead_R, UR, (lambda X: tr(X, UR, U[-1]),)))


def fp64_uncertainty(dev, E, eta, T_ref, n_gauges=2, seed=1234):
    rng = np.random.default_rng(seed)
    d = np.zeros_like(T_ref)
    for _ in range(n_gauges):
        d = np.maximum(d, np.abs(o.transmission(gauge_transform(dev, rng), E, eta) - T_ref))
    return d


def fp64_bar(T_ref, spread=None):
    bar = FP64_REL * np.maximum(np.abs(T_ref), 1e-6)
    if spread is not None:
        bar = np.maximum(bar, 4.0 * spread)
    return bar
