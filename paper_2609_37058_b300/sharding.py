"""Energy-wave sharding across ranks (one GPU per rank).

Energies are independent, so a multi-GPU job splits the energy grid into
waves of W energies and deals them round-robin to ranks; every rank runs its
own plan on its own GPU and the only exchange is the final host-side gather
of T(E).  No collective runs inside the transport path.
"""
from __future__ import annotations


def wave_bounds(n_E: int, W: int, k: int) -> tuple[int, int]:
    """(start, count) of global wave k of a grid of n_E energies."""
    if W <= 0 or n_E <= 0:
        raise ValueError("need W > 0 and n_E > 0")
    n_waves = (n_E + W - 1) // W
    k %= n_waves
    start = k * W
    return start, min(W, n_E - start)


def rank_waves(n_E: int, W: int, rank: int, world: int) -> list[tuple[int, int]]:
    """Waves of one full pass over the grid owned by `rank` of `world`."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    n_waves = (n_E + W - 1) // W
    return [wave_bounds(n_E, W, k) for k in range(rank, n_waves, world)]


def step_wave(n_E: int, W: int, rank: int, world: int, step: int) -> tuple[int, int]:
    """Wave processed by `rank` at benchmark step `step` (wraps around)."""
    return wave_bounds(n_E, W, step * world + rank)


def gather_transmission(T_local, waves, n_E, group=None):
    """Assemble the full T(E) on every rank from each rank's waves (host
    tensors).  Uses torch.distributed.all_gather_object: a host-side gather
    after the transport work, not part of it."""
    import numpy as np
    import torch.distributed as dist
    pieces = [(s, np.asarray(T_local[i:i + c])) for i, (s, c) in zip(_offsets(waves), waves)]
    out = [None] * dist.get_world_size(group)
    dist.all_gather_object(out, pieces, group=group)
    T = np.full(n_E, np.nan)
    for rank_pieces in out:
        for s, arr in rank_pieces:
            T[s:s + len(arr)] = arr
    return T


def _offsets(waves):
    off, res = 0, []
    for _, c in waves:
        res.append(off)
        off += c
    return res
