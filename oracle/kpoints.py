"""FP64 CPU oracle for transverse k-point sampling.  TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import or run this module; the CUDA library shares no code
with it.

The paper states the RGF cost per energy point and per transverse k-point
(Results, the scaling paragraph) and samples the transverse Brillouin zone
with Monkhorst-Pack meshes (Methods, transport paragraph).  For a device
periodic in the transverse directions with blocks X(R) between the home cell
and the cell displaced by the lattice vector R:

* X(k) = sum_R exp(2 pi i k.R) X(R) for every block (k fractional, R integer);
* T(E, k) is the transmission of the k-resolved device (``rgf_oracle``);
* the transmission per transverse cell is the weighted mean over the mesh,
  T(E) = sum_k w_k T(E, k), sum_k w_k = 1.

Pins (``tests/test_oracle_kpoints.py``): a stack of uniform chains with
transverse hopping, whose T(E, k) is the chain closed form at the shifted
on-site energy eps + 2 ty cos(2 pi k); and the exact identity between the
M-point mesh k = m/M and the real-space ring of M transverse cells,
T_ring(E) = sum_m T(E, m/M), with the ring built here from its definition.
"""
from __future__ import annotations

import numpy as np

from . import rgf_oracle
from synth.devices import Device, Lead


def phases(R, k):
    """exp(2 pi i k.R_r) for every lattice vector R_r."""
    R = np.asarray(R, dtype=np.float64)
    return np.exp(2j * np.pi * (R @ np.asarray(k, dtype=np.float64)))


def bloch_sum(X_R, R, k):
    """sum_r phase_r X_R[r] (X_R has the lattice-vector axis first)."""
    p = phases(R, k)
    return np.tensordot(p, np.asarray(X_R), axes=(0, 0))


def device_at_k(kdev, k) -> Device:
    """The k-resolved device: every block (and lead block) Bloch-summed."""
    bs = lambda X: np.ascontiguousarray(bloch_sum(X, kdev.R, k))
    lead = lambda L: Lead(bs(L.H00), bs(L.S00), bs(L.H10), bs(L.S10), bs(L.Hc), bs(L.Sc))
    return Device(H_diag=bs(kdev.H_diag), S_diag=bs(kdev.S_diag), H_lower=bs(kdev.H_lower),
                  S_lower=bs(kdev.S_lower), lead_L=lead(kdev.lead_L), lead_R=lead(kdev.lead_R),
                  name=f"{kdev.name}@k={tuple(np.round(k, 6))}")


def transmission_kmesh(kdev, kpts, weights, energies, eta, **kw):
    """(T(E) averaged with the weights, T(E, k) per k-point)."""
    Tk = np.array([rgf_oracle.transmission(device_at_k(kdev, k), energies, eta, **kw) for k in kpts])
    return np.tensordot(np.asarray(weights, dtype=np.float64), Tk, axes=(0, 0)), Tk


def ring_device(kdev, M: int) -> Device:
    """M transverse cells closed into a ring (one periodic direction, R along
    the first lattice axis): block (m, m') of every layer is the sum of X(R)
    over the R with m' - m = R1 (mod M).  Block size b*M."""
    if np.any(kdev.R[:, 1] != 0):
        raise ValueError("ring_device handles one periodic direction")
    b = kdev.b

    def ring(X):  # X: (n_R, n_blocks, b, b) -> (n_blocks, bM, bM)
        nbl = X.shape[1]
        out = np.zeros((nbl, b * M, b * M), dtype=np.complex128)
        for r, (R1, _) in enumerate(kdev.R):
            for m in range(M):
                mp = (m + int(R1)) % M
                out[:, m * b:(m + 1) * b, mp * b:(mp + 1) * b] += X[r]
        return out

    def ring1(X):  # lead blocks (n_R, b, b)
        return ring(np.asarray(X)[:, None])[0]

    lead = lambda L: Lead(ring1(L.H00), ring1(L.S00), ring1(L.H10), ring1(L.S10), ring1(L.Hc), ring1(L.Sc))
    return Device(H_diag=ring(kdev.H_diag), S_diag=ring(kdev.S_diag), H_lower=ring(kdev.H_lower),
                  S_lower=ring(kdev.S_lower), lead_L=lead(kdev.lead_L), lead_R=lead(kdev.lead_R),
                  name=f"{kdev.name}_ring{M}")
