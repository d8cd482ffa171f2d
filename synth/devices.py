"""Seeded synthetic block-tridiagonal nonorthogonal devices.

Layout convention (shared by every consumer, stated once here):

* A device has ``N`` principal layers of block size ``b``.  The Hamiltonian
  H and overlap S are block tridiagonal and Hermitian.
* ``H_diag[i]`` = H_{i,i} and ``S_diag[i]`` = S_{i,i}, i = 0..N-1.
* ``H_lower[i-1]`` = H_{i,i-1} and ``S_lower[i-1]`` = S_{i,i-1}, i = 1..N-1
  (the block whose row layer is to the right of its column layer).  The
  upper blocks follow by Hermiticity, H_{i-1,i} = H_{i,i-1}^dagger.
* A lead is a semi-infinite periodic chain of principal layers.  ``H00``,
  ``S00`` are the on-site blocks of one lead cell; ``H10``, ``S10`` couple
  consecutive lead cells in the same left-to-right orientation as the device
  (row cell to the right of column cell); ``Hc``, ``Sc`` couple the lead to
  the device, again row-right/column-left: for the left lead Hc = H_{0,-1},
  for the right lead Hc = H_{N,N-1}.
* All blocks are complex128, row-major.

Entry law: a complex "N(0, s)" entry is s * (x + i y) / sqrt(2) with x, y
independent standard normals (so its absolute variance is s^2).  The random
stream is numpy's PCG64 seeded with the workload seed; the draw order is:
all A (N,b,b), all B (N,b,b), all coupling-H draws (N-1,b,b), all
coupling-S draws (N-1,b,b), then dopant layers, dopant orbitals and dopant
shifts.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Lead:
    H00: np.ndarray
    S00: np.ndarray
    H10: np.ndarray
    S10: np.ndarray
    Hc: np.ndarray
    Sc: np.ndarray


@dataclasses.dataclass
class Device:
    H_diag: np.ndarray   # (N, b, b)
    S_diag: np.ndarray   # (N, b, b)
    H_lower: np.ndarray  # (N-1, b, b)
    S_lower: np.ndarray  # (N-1, b, b)
    lead_L: Lead
    lead_R: Lead
    name: str = ""

    @property
    def n_layers(self) -> int:
        return self.H_diag.shape[0]

    @property
    def b(self) -> int:
        return self.H_diag.shape[1]

    def nbytes(self) -> int:
        return int(self.H_diag.nbytes + self.S_diag.nbytes + self.H_lower.nbytes + self.S_lower.nbytes)


def _cnormal(rng: np.random.Generator, shape, s: float) -> np.ndarray:
    x = rng.standard_normal(tuple(shape) + (2,))
    return (s / math.sqrt(2.0)) * (x[..., 0] + 1j * x[..., 1])


def _herm(m: np.ndarray) -> np.ndarray:
    return 0.5 * (m + np.conj(np.swapaxes(m, -1, -2)))


def _dag(m: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(np.conj(np.swapaxes(m, -1, -2)))


def periodic_leads(H_diag, S_diag, H_lower, S_lower):
    """Leads that continue the first and last device layers periodically.

    Left lead: every cell is a copy of layer 0 and consecutive cells (and the
    lead-device link) are coupled like layers 0 and 1.  Right lead: copies of
    layer N-1, coupled like layers N-2 and N-1.  For a one-layer device the
    couplings must be supplied separately, so N >= 2 here.
    """
    N = H_diag.shape[0]
    if N < 2:
        raise ValueError("periodic leads need at least two layers")
    lead_L = Lead(H00=H_diag[0].copy(), S00=S_diag[0].copy(),
                  H10=H_lower[0].copy(), S10=S_lower[0].copy(),
                  Hc=H_lower[0].copy(), Sc=S_lower[0].copy())
    lead_R = Lead(H00=H_diag[N - 1].copy(), S00=S_diag[N - 1].copy(),
                  H10=H_lower[N - 2].copy(), S10=S_lower[N - 2].copy(),
                  Hc=H_lower[N - 2].copy(), Sc=S_lower[N - 2].copy())
    return lead_L, lead_R


def random_device(N: int, b: int, seed: int, *, metal_frac: float = 0.0,
                  gap_offset: float = 0.0, n_dopant_layers: int = 0,
                  dopant_orbitals: int = 13, dopant_mu: float = -0.3,
                  dopant_sigma: float = 0.1, name: str = "") -> Device:
    """Draw one metal-channel-metal junction.

    * On-site: H_ii = (A + A^dagger)/2 with A entries N(0, 1/sqrt(b));
      S_ii = I + 0.05 (B + B^dagger)/2 with B drawn like A.
    * Layers i < round(metal_frac*N) and i >= N - round(metal_frac*N) are
      metal; the rest are channel.  A coupling H_{i,i+1} has entries
      N(0, 1/sqrt(b)) when both layers are metal, else N(0, 0.5/sqrt(b)).
      S_{i,i+1} entries are N(0, 0.02*sqrt(8/b)) (N(0, 0.02) at b = 8).
    * Channel layers get +gap_offset on orbitals [0, b/2) and -gap_offset on
      [b/2, b) of the H_ii diagonal.
    * ``n_dopant_layers`` distinct channel layers each get shifts
      N(dopant_mu, dopant_sigma) (real) on ``dopant_orbitals`` distinct
      diagonal entries of H_ii.
    * Both leads are periodic continuations of the end layers.
    """
    if N < 2 or b < 1:
        raise ValueError("need N >= 2 and b >= 1")
    rng = np.random.default_rng(seed)
    n_metal = int(round(metal_frac * N))
    metal = np.zeros(N, dtype=bool)
    if n_metal > 0:
        metal[:n_metal] = True
        metal[N - n_metal:] = True

    A = _cnormal(rng, (N, b, b), 1.0 / math.sqrt(b))
    B = _cnormal(rng, (N, b, b), 1.0 / math.sqrt(b))
    C = _cnormal(rng, (N - 1, b, b), 1.0)
    D = _cnormal(rng, (N - 1, b, b), 0.02 * math.sqrt(8.0 / b))

    H_diag = _herm(A)
    S_diag = np.eye(b)[None, :, :] + 0.05 * _herm(B)
    both_metal = metal[:-1] & metal[1:]
    scale = np.where(both_metal, 1.0, 0.5) / math.sqrt(b)
    H_upper = C * scale[:, None, None]
    S_upper = D

    if gap_offset != 0.0:
        off = np.concatenate([np.full(b // 2, gap_offset), np.full(b - b // 2, -gap_offset)])
        for i in np.nonzero(~metal)[0]:
            H_diag[i][np.diag_indices(b)] += off

    if n_dopant_layers > 0:
        channel = np.nonzero(~metal)[0]
        if n_dopant_layers > channel.size:
            raise ValueError("more dopant layers than channel layers")
        k = min(dopant_orbitals, b)
        layers = rng.choice(channel, size=n_dopant_layers, replace=False)
        for i in layers:
            orbs = rng.choice(b, size=k, replace=False)
            shifts = dopant_mu + dopant_sigma * rng.standard_normal(k)
            H_diag[i][orbs, orbs] += shifts

    H_lower = _dag(H_upper)
    S_lower = _dag(S_upper)
    lead_L, lead_R = periodic_leads(H_diag, S_diag, H_lower, S_lower)
    return Device(H_diag=np.ascontiguousarray(H_diag), S_diag=np.ascontiguousarray(S_diag),
                  H_lower=H_lower, S_lower=S_lower, lead_L=lead_L, lead_R=lead_R, name=name)


def chain_device(N: int, eps: float = 0.0, t: float = 1.0) -> Device:
    """Uniform nearest-neighbour chain: b = 1, on-site eps, hopping t, S = I.

    Both leads are the same chain continued to infinity, so the device is a
    window of N sites cut out of a perfect infinite chain.
    """
    H_diag = np.full((N, 1, 1), eps, dtype=np.complex128)
    S_diag = np.ones((N, 1, 1), dtype=np.complex128)
    H_lower = np.full((max(N - 1, 0), 1, 1), t, dtype=np.complex128)
    S_lower = np.zeros((max(N - 1, 0), 1, 1), dtype=np.complex128)
    one = np.ones((1, 1), dtype=np.complex128)
    zero = np.zeros((1, 1), dtype=np.complex128)
    lead = lambda: Lead(H00=eps * one, S00=one.copy(), H10=t * one, S10=zero.copy(),
                        Hc=t * one, Sc=zero.copy())
    return Device(H_diag=H_diag, S_diag=S_diag, H_lower=H_lower, S_lower=S_lower,
                  lead_L=lead(), lead_R=lead(), name=f"chain_N{N}")


def energy_grid(lo: float, hi: float, n: int) -> np.ndarray:
    """Uniform real energies, both endpoints included."""
    return np.linspace(lo, hi, n, dtype=np.float64)


# Named workloads: the junction shapes of the paper's Pt-Si-Pt / Pt-Si:P-Pt
# devices, drawn synthetically.
WORKLOADS = {
    "chain_N64": dict(kind="chain", N=64, b=1, n_E=256, E_lo=-3.0, E_hi=3.0, eta=1e-6),
    "small_N64_b8": dict(kind="random", N=64, b=8, n_E=256, E_lo=-3.0, E_hi=3.0, eta=1e-6,
                         seed=0, metal_frac=0.0, gap_offset=0.0, n_dopant_layers=0),
    "junction_N200_b128": dict(kind="random", N=200, b=128, n_E=1024, E_lo=-2.0, E_hi=2.0,
                               eta=1e-5, seed=1, metal_frac=0.25, gap_offset=0.6,
                               n_dopant_layers=0),
    "doped_N500_b256": dict(kind="random", N=500, b=256, n_E=2048, E_lo=-1.5, E_hi=1.5,
                            eta=1e-6, seed=2, metal_frac=0.25, gap_offset=0.6,
                            n_dopant_layers=5),
}


def make_device(name: str, **override) -> Device:
    w = dict(WORKLOADS[name])
    w.update(override)
    if w["kind"] == "chain":
        return chain_device(w["N"])
    return random_device(w["N"], w["b"], w["seed"], metal_frac=w["metal_frac"],
                         gap_offset=w["gap_offset"], n_dopant_layers=w["n_dopant_layers"],
                         name=name)


def make_workload(name: str, **override):
    """Return (device, energies, eta) for a named workload."""
    w = dict(WORKLOADS[name])
    w.update(override)
    dev = make_device(name, **override)
    return dev, energy_grid(w["E_lo"], w["E_hi"], w["n_E"]), float(w["eta"])


def uneven_batch(n_dev: int, seed: int, *, N_lo: int, N_hi: int, b_choices, n_E: int,
                 E_lo: float = -2.0, E_hi: float = 2.0, eta: float = 1e-5,
                 metal_frac: float = 0.25, gap_offset: float = 0.6):
    """Devices of uneven length and block size for batched runs.

    Lengths are log-uniform in [N_lo, N_hi] (integers), block sizes drawn
    uniformly from ``b_choices``, every device a metal-channel-metal junction
    of the ``junction_N200_b128`` kind with its own seed.  Draw order: the N
    values, then the b values, then the per-device seeds, all from one
    ``default_rng(seed)``.  Returns a list of (device, energies, eta).
    """
    rng = np.random.default_rng(seed)
    Ns = np.exp(rng.uniform(math.log(N_lo), math.log(N_hi + 1), n_dev)).astype(np.int64)
    Ns = np.clip(Ns, max(N_lo, 2), N_hi)
    bs = rng.choice(np.asarray(b_choices, dtype=np.int64), size=n_dev)
    seeds = rng.integers(0, 2**31 - 1, size=n_dev)
    out = []
    for N, b, s in zip(Ns, bs, seeds):
        n_metal = int(round(metal_frac * int(N)))
        mf = metal_frac if 0 < n_metal < int(N) / 2 else 0.0
        dev = random_device(int(N), int(b), int(s), metal_frac=mf, gap_offset=gap_offset,
                            name=f"uneven_N{int(N)}_b{int(b)}")
        out.append((dev, energy_grid(E_lo, E_hi, n_E), float(eta)))
    return out


def serving_trace(seed: int, *, rate: float, duration: float, N_lo: int, N_hi: int, b_lo: int,
                  b_hi: int, nE_lo: int, nE_hi: int, window: float = 1.5, eta: float = 1e-5):
    """Poisson arrivals of transport requests.

    Inter-arrival times are exponential with mean 1/rate until ``duration``
    seconds; each request draws a length log-uniform in [N_lo, N_hi], a block
    size uniform in [b_lo, b_hi], a number of energies uniform in
    [nE_lo, nE_hi] and an energy window [c - window, c + window] with its
    centre c uniform in [-0.5, 0.5].  Returns a list of dicts (t, N, b, n_E,
    E, eta, seed).  Devices are not drawn here.
    """
    rng = np.random.default_rng(seed)
    out = []
    t = 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        N = int(np.clip(np.exp(rng.uniform(math.log(N_lo), math.log(N_hi + 1))), max(N_lo, 2), N_hi))
        b = int(rng.integers(b_lo, b_hi + 1))
        n_E = int(rng.integers(nE_lo, nE_hi + 1))
        c = float(rng.uniform(-0.5, 0.5))
        out.append(dict(t=t, N=N, b=b, n_E=n_E, E=energy_grid(c - window, c + window, n_E), eta=eta,
                        seed=int(rng.integers(0, 2**31 - 1))))
    return out


@dataclasses.dataclass
class KDevice:
    """A device periodic in the transverse directions: every block is given
    per transverse lattice vector R (integer coordinates, row r of ``R``);
    leads likewise (each Lead field has shape (n_R, b, b)).  X[r] is the
    block between the home cell and the cell displaced by R[r]."""
    R: np.ndarray        # (n_R, 2) int
    H_diag: np.ndarray   # (n_R, N, b, b)
    S_diag: np.ndarray
    H_lower: np.ndarray  # (n_R, N-1, b, b)
    S_lower: np.ndarray
    lead_L: Lead
    lead_R: Lead
    name: str = ""

    @property
    def n_layers(self) -> int:
        return self.H_diag.shape[1]

    @property
    def b(self) -> int:
        return self.H_diag.shape[2]


def periodic_kdevice(N: int, b: int, seed: int, *, metal_frac: float = 0.25, gap_offset: float = 0.6,
                     transverse: float = 0.3, name: str = "") -> KDevice:
    """Junction with one periodic transverse direction, R in {0, +1, -1}.

    R = 0 blocks follow ``random_device`` (same recipe and seed).  The
    transverse blocks are drawn afterwards from the same generator, in this
    order: on-site H_ii(+1) entries N(0, transverse/sqrt(b)); S_ii(+1)
    entries N(0, 0.01 sqrt(8/b)); couplings H_{i,i-1}(+1) and H_{i,i-1}(-1)
    entries N(0, 0.5 transverse/sqrt(b)); S_{i,i-1}(+1) and S_{i,i-1}(-1)
    entries N(0, 0.005 sqrt(8/b)).  On-site blocks satisfy X(-1) = X(+1)^dagger
    (so that H(k) and S(k) are Hermitian).  Leads repeat layer 0 and layer
    N-1 as in ``periodic_leads``.
    """
    d0 = random_device(N, b, seed, metal_frac=metal_frac, gap_offset=gap_offset)
    rng = np.random.default_rng([seed, 1])
    Hd1 = _cnormal(rng, (N, b, b), transverse / math.sqrt(b))
    Sd1 = _cnormal(rng, (N, b, b), 0.01 * math.sqrt(8.0 / b))
    Hl = [_cnormal(rng, (N - 1, b, b), 0.5 * transverse / math.sqrt(b)) for _ in range(2)]
    Sl = [_cnormal(rng, (N - 1, b, b), 0.005 * math.sqrt(8.0 / b)) for _ in range(2)]
    R = np.array([[0, 0], [1, 0], [-1, 0]], dtype=np.int32)
    H_diag = np.stack([d0.H_diag, Hd1, _dag(Hd1)])
    S_diag = np.stack([d0.S_diag, Sd1, _dag(Sd1)])
    H_lower = np.stack([d0.H_lower, Hl[0], Hl[1]])
    S_lower = np.stack([d0.S_lower, Sl[0], Sl[1]])
    lead = lambda i, j: Lead(H00=H_diag[:, i].copy(), S00=S_diag[:, i].copy(), H10=H_lower[:, j].copy(),
                             S10=S_lower[:, j].copy(), Hc=H_lower[:, j].copy(), Sc=S_lower[:, j].copy())
    return KDevice(R=R, H_diag=np.ascontiguousarray(H_diag), S_diag=np.ascontiguousarray(S_diag),
                   H_lower=np.ascontiguousarray(H_lower), S_lower=np.ascontiguousarray(S_lower),
                   lead_L=lead(0, 0), lead_R=lead(N - 1, N - 2), name=name or f"kdev_N{N}_b{b}")


def chain_stack(N: int, eps: float = 0.0, t: float = 1.0, ty: float = 0.25) -> KDevice:
    """Uniform chains (on-site eps, hopping t along transport, S = I) side by
    side, each coupled to its transverse neighbours by ty: b = 1, R in
    {0, +1, -1}, H_ii(+-1) = ty.  Leads continue the chains."""
    R = np.array([[0, 0], [1, 0], [-1, 0]], dtype=np.int32)
    z = lambda *s: np.zeros(s, dtype=np.complex128)
    H_diag, S_diag = z(3, N, 1, 1), z(3, N, 1, 1)
    H_diag[0], H_diag[1], H_diag[2] = eps, ty, ty
    S_diag[0] = 1.0
    H_lower, S_lower = z(3, N - 1, 1, 1), z(3, N - 1, 1, 1)
    H_lower[0] = t
    lead = lambda: Lead(H00=H_diag[:, 0].copy(), S00=S_diag[:, 0].copy(), H10=H_lower[:, 0].copy(),
                        S10=S_lower[:, 0].copy(), Hc=H_lower[:, 0].copy(), Sc=S_lower[:, 0].copy())
    return KDevice(R=R, H_diag=H_diag, S_diag=S_diag, H_lower=H_lower, S_lower=S_lower, lead_L=lead(),
                   lead_R=lead(), name=f"chain_stack_N{N}")


def monkhorst_pack(n1: int, n2: int = 1):
    """Monkhorst-Pack mesh: k_i = (2 m - n_i - 1) / (2 n_i), m = 1..n_i,
    equal weights.  Returns (k (n, 2), w (n,))."""
    k1 = (2.0 * np.arange(1, n1 + 1) - n1 - 1) / (2.0 * n1)
    k2 = (2.0 * np.arange(1, n2 + 1) - n2 - 1) / (2.0 * n2)
    k = np.array([[a, b_] for a in k1 for b_ in k2], dtype=np.float64)
    return k, np.full(k.shape[0], 1.0 / k.shape[0])


def random_phase_vectors(n_vec: int, n: int, seed: int) -> np.ndarray:
    """Random vectors for stochastic trace estimates: n_vec vectors of n
    entries exp(2 pi i u), u uniform in [0, 1) (so E[r r^dag] = I and every
    |r_j| = 1), numpy PCG64 seeded with ``seed``; shape (n_vec, n)."""
    rng = np.random.default_rng(seed)
    return np.exp(2j * np.pi * rng.random((n_vec, n)))
