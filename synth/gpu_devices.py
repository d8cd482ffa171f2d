"""Seeded synthetic junctions drawn directly in device memory (torch).

Same recipe as ``devices.random_device`` (on-site Hermitian blocks with
N(0, 1/sqrt(b)) entries, S_ii = I + 0.05 Hermitian noise, couplings
N(0, 1/sqrt(b)) between metal layers and N(0, 0.5/sqrt(b)) elsewhere,
S couplings N(0, 0.02 sqrt(8/b)), gap offsets on channel layers, periodic
leads), drawn with torch's generator on the GPU so that batches of tens of
GB never pass through host memory.  The numbers differ from the numpy draw
of the same seed; ``to_host`` returns a ``devices.Device`` for the oracle.
Holds no transport arithmetic.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from .devices import Device, Lead


@dataclasses.dataclass
class GpuDevice:
    H_diag: object  # torch complex128 (N, b, b) on the GPU
    S_diag: object
    H_lower: object  # (N-1, b, b)
    S_lower: object
    lead_L: tuple    # (H00, S00, H10, S10, Hc, Sc) views
    lead_R: tuple
    name: str = ""

    @property
    def n_layers(self) -> int:
        return int(self.H_diag.shape[0])

    @property
    def b(self) -> int:
        return int(self.H_diag.shape[1])

    def nbytes(self) -> int:
        return int(sum(t.numel() * 16 for t in (self.H_diag, self.S_diag, self.H_lower, self.S_lower)))

    def to_host(self) -> Device:
        c = lambda t: t.detach().cpu().numpy().copy()
        lead = lambda L: Lead(*(c(x) for x in L))
        return Device(H_diag=c(self.H_diag), S_diag=c(self.S_diag), H_lower=c(self.H_lower),
                      S_lower=c(self.S_lower), lead_L=lead(self.lead_L), lead_R=lead(self.lead_R),
                      name=self.name)


def random_device_gpu(N: int, b: int, seed: int, *, metal_frac: float = 0.0, gap_offset: float = 0.0,
                      device: str = "cuda") -> GpuDevice:
    import torch

    if N < 2 or b < 1:
        raise ValueError("need N >= 2 and b >= 1")
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    f64 = torch.float64

    def cnormal(shape, s):
        x = torch.randn(tuple(shape) + (2,), generator=g, device=device, dtype=f64)
        return torch.view_as_complex(x) * (s / math.sqrt(2.0))

    def herm(m):
        return 0.5 * (m + m.conj().transpose(-1, -2))

    n_metal = int(round(metal_frac * N))
    metal = torch.zeros(N, dtype=torch.bool)
    if n_metal > 0:
        metal[:n_metal] = True
        metal[N - n_metal:] = True
    H_diag = herm(cnormal((N, b, b), 1.0 / math.sqrt(b)))
    S_diag = herm(cnormal((N, b, b), 1.0 / math.sqrt(b))) * 0.05
    S_diag.diagonal(dim1=-2, dim2=-1).add_(1.0)
    both = (metal[:-1] & metal[1:]).to(device)
    scale = torch.where(both, 1.0, 0.5).to(f64) / math.sqrt(b)
    H_upper = cnormal((N - 1, b, b), 1.0) * scale[:, None, None]
    S_upper = cnormal((N - 1, b, b), 0.02 * math.sqrt(8.0 / b))
    if gap_offset != 0.0:
        off = torch.cat([torch.full((b // 2,), gap_offset, dtype=f64),
                         torch.full((b - b // 2,), -gap_offset, dtype=f64)]).to(device)
        ch = torch.nonzero(~metal).flatten().to(device)
        H_diag[ch] += torch.diag_embed(off).to(H_diag.dtype)
    H_lower = H_upper.conj().transpose(-1, -2).contiguous()
    S_lower = S_upper.conj().transpose(-1, -2).contiguous()
    del H_upper, S_upper
    H_diag, S_diag = H_diag.contiguous(), S_diag.contiguous()
    lead_L = (H_diag[0], S_diag[0], H_lower[0], S_lower[0], H_lower[0], S_lower[0])
    lead_R = (H_diag[N - 1], S_diag[N - 1], H_lower[N - 2], S_lower[N - 2], H_lower[N - 2], S_lower[N - 2])
    return GpuDevice(H_diag, S_diag, H_lower, S_lower, lead_L, lead_R, name=f"gpu_N{N}_b{b}_s{seed}")


def uneven_shapes(n_dev: int, seed: int, *, N_lo: int, N_hi: int, b_choices):
    """(N, b, seed) triples: N log-uniform in [N_lo, N_hi], b from b_choices."""
    rng = np.random.default_rng(seed)
    Ns = np.clip(np.exp(rng.uniform(math.log(N_lo), math.log(N_hi + 1), n_dev)).astype(np.int64),
                 max(N_lo, 2), N_hi)
    bs = rng.choice(np.asarray(b_choices, dtype=np.int64), size=n_dev)
    seeds = rng.integers(0, 2**31 - 1, size=n_dev)
    return [(int(N), int(b), int(s)) for N, b, s in zip(Ns, bs, seeds)]
