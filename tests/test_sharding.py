"""Energy-wave sharding across ranks: coverage, and a world_size-2 gloo run
of the host-side gather and of the max-over-ranks timing reduction."""
import os
import socket

import numpy as np
import pytest

from paper_2609_37058_b300.sharding import rank_waves, step_wave, wave_bounds


@pytest.mark.parametrize("n_E,W,world", [(2048, 148, 1), (2048, 148, 2), (2048, 148, 8), (37, 5, 3), (5, 8, 2)])
def test_waves_cover_grid_once(n_E, W, world):
    seen = np.zeros(n_E, dtype=int)
    for r in range(world):
        for s, c in rank_waves(n_E, W, r, world):
            seen[s:s + c] += 1
    assert np.all(seen == 1)


def test_step_waves_are_disjoint_across_ranks():
    n_E, W, world = 2048, 148, 4
    for step in range(3):
        starts = [step_wave(n_E, W, r, world, step)[0] for r in range(world)]
        assert len(set(starts)) == world
    assert wave_bounds(2048, 148, 13) == (1924, 124)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n_E, W, q):
    import torch
    import torch.distributed as dist
    from paper_2609_37058_b300.sharding import gather_transmission, rank_waves
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    E = np.linspace(-1.5, 1.5, n_E)
    waves = rank_waves(n_E, W, rank, world)
    # Stand-in per-energy result computed by this rank only.
    T_local = np.concatenate([np.cos(E[s:s + c]) for s, c in waves])
    T = gather_transmission(T_local, waves, n_E)
    t = torch.tensor([1.0 + rank])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    q.put((rank, bool(np.allclose(T, np.cos(E))), float(t.item())))
    dist.destroy_process_group()


def test_gloo_world2_gather_and_max():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, 101, 7, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
    assert all(ok for _, ok, _ in res)
    assert all(m == 2.0 for _, _, m in res)
