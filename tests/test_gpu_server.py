"""Multi-device server (batching of uneven devices, serving) through the C ABI.

Every request's T(E) is checked against the FP64 oracle (|dT| <= 1e-6
absolute, the mixed-precision bar), a request's result alone and inside a
mix of others is compared, and admission by resident bytes is exercised.
"""
import numpy as np
import pytest

from helpers import MIXED_ABS
from oracle import rgf_oracle as o
from synth import Lead, random_device
from synth.devices import Device, energy_grid, uneven_batch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rgf():
    from paper_2609_37058_b300 import build, rgf as r
    build.build()
    return r


def one_layer_device(b, seed):
    """N = 1: the single layer of a two-layer junction, leads unchanged."""
    d = random_device(2, b, seed)
    return Device(H_diag=d.H_diag[:1].copy(), S_diag=d.S_diag[:1].copy(),
                  H_lower=np.zeros((0, b, b), complex), S_lower=np.zeros((0, b, b), complex),
                  lead_L=d.lead_L, lead_R=d.lead_R, name="one_layer")


def serve(rgf, jobs, **opt):
    with rgf.Server(**opt) as sv:
        tickets = [sv.submit(d, E, eta) for d, E, eta in jobs]
        res = [sv.poll(t, timeout_us=300_000_000) for t in tickets]
        stats = sv.stats()
    assert all(r is not None for r in res), "a request did not complete within 300 s"
    return res, stats


def test_uneven_devices_match_oracle(rgf):
    # Lengths 2..14, block sizes 5..16 (padded to multiples of 8), more items
    # than slots, so that slots are refilled across devices.
    jobs = uneven_batch(6, 7, N_lo=2, N_hi=14, b_choices=[5, 8, 12, 16], n_E=12, eta=1e-5)
    jobs.append((one_layer_device(6, 3), energy_grid(-1.0, 1.0, 5), 1e-5))
    res, stats = serve(rgf, jobs, slots=16, class_step=8)
    assert stats["completed"] == len(jobs) and stats["energies_done"] == sum(len(E) for _, E, _ in jobs)
    assert stats["engines"] == len({-(-d.b // 8) * 8 for d, _, _ in jobs})
    for (dev, E, eta), (T, err, flags, lat) in zip(jobs, res):
        T_o = o.transmission(dev, E, eta)
        assert np.all((flags & ~rgf.RGF_FLAG_REFINE) == 0), (dev.name, flags)
        assert np.abs(T - T_o).max() <= MIXED_ABS, (dev.name, np.abs(T - T_o).max())
        assert lat > 0


def test_result_alone_equals_result_in_mix(rgf):
    target = random_device(9, 12, 11, metal_frac=0.25, gap_offset=0.6)
    E = energy_grid(-1.5, 1.5, 20)
    alone, _ = serve(rgf, [(target, E, 1e-6)], slots=8, class_step=8)
    others = uneven_batch(5, 12, N_lo=2, N_hi=20, b_choices=[8, 12, 16], n_E=17, eta=1e-6)
    mix = others[:2] + [(target, E, 1e-6)] + others[2:]
    mixed, stats = serve(rgf, mix, slots=8, class_step=8)
    T_alone, T_mix = alone[0][0], mixed[2][0]
    # Each item runs the same per-entry operations in any mix.
    assert np.abs(T_alone - T_mix).max() <= MIXED_ABS
    assert np.array_equal(alone[0][2], mixed[2][2])
    assert stats["completed"] == len(mix)
    T_o = o.transmission(target, E, 1e-6)
    assert np.abs(T_mix - T_o).max() <= MIXED_ABS


def test_padding_leaves_T_unchanged(rgf):
    dev = random_device(6, 10, 5)
    E = energy_grid(-2.0, 2.0, 16)
    (r1,), _ = serve(rgf, [(dev, E, 1e-5)], slots=8, class_step=1)
    (r2,), _ = serve(rgf, [(dev, E, 1e-5)], slots=8, class_step=32)
    assert np.abs(r1[0] - r2[0]).max() <= 1e-9
    assert np.abs(r1[0] - o.transmission(dev, E, 1e-5)).max() <= MIXED_ABS


def test_admission_by_resident_bytes(rgf):
    jobs = uneven_batch(5, 21, N_lo=4, N_hi=12, b_choices=[16], n_E=6, eta=1e-5)
    nn = 16 * 16
    need = [(4 * d.n_layers - 2) * nn * 16 + 12 * nn * 16 for d, _, _ in jobs]
    cap = max(need) + 1024  # one request at a time
    res, stats = serve(rgf, jobs, slots=8, class_step=16, capacity_bytes=cap)
    assert stats["completed"] == len(jobs)
    assert stats["peak_resident_bytes"] <= cap
    for (dev, E, eta), (T, err, flags, lat) in zip(jobs, res):
        assert np.abs(T - o.transmission(dev, E, eta)).max() <= MIXED_ABS
    # A request that could never fit is rejected at submission.
    with rgf.Server(slots=8, class_step=16, capacity_bytes=1 << 16) as sv:
        with pytest.raises(rgf.RGFError) as ex:
            sv.submit(*jobs[0])
        assert ex.value.status == rgf.RGF_E_REJECTED
        assert sv.stats()["rejected"] == 1


def test_poll_timeout_and_not_ready(rgf):
    jobs = uneven_batch(1, 5, N_lo=30, N_hi=30, b_choices=[32], n_E=4, eta=1e-5)
    with rgf.Server(slots=8, class_step=32) as sv:
        t = sv.submit(*jobs[0])
        # A zero timeout returns at once, done or not.
        r = sv.poll(t, timeout_us=0)
        if r is None:
            r = sv.poll(t, timeout_us=300_000_000)
        assert r is not None and np.all(np.isfinite(r[0]))


def test_concurrent_engines_with_large_blocks(rgf):
    # Several block-size engines whose inverses need more than 48 KB of
    # shared memory run at the same time on their own host threads.
    jobs = [(random_device(3, b, 40 + i), energy_grid(-1.0, 1.0, 6), 1e-5)
            for i, b in enumerate([192, 224, 256, 160, 200])]
    res, stats = serve(rgf, jobs, slots=8, class_step=32)
    assert stats["engines"] == 4
    for (dev, E, eta), (T, err, flags, lat) in zip(jobs, res):
        assert np.abs(T - o.transmission(dev, E, eta)).max() <= MIXED_ABS, dev.b


def test_graph_replay_matches_direct_launches(rgf, monkeypatch):
    # Steps from the third on replay a captured CUDA graph; the same items
    # launched directly (no graphs, host-side reseed decision) agree.
    jobs = uneven_batch(3, 31, N_lo=6, N_hi=15, b_choices=[12, 24], n_E=9, eta=1e-6)
    with_graphs, st = serve(rgf, jobs, slots=8, class_step=8)
    monkeypatch.setenv("RGF_NO_GRAPHS", "1")
    direct, _ = serve(rgf, jobs, slots=8, class_step=8)
    assert st["steps"] > 2
    for (dev, E, eta), a, b in zip(jobs, with_graphs, direct):
        assert np.abs(a[0] - b[0]).max() <= 1e-12
        assert np.abs(a[0] - o.transmission(dev, E, eta)).max() <= MIXED_ABS


def test_class_settings_give_the_same_result(rgf):
    # Tile width and panel width change how the work is cut, not what each
    # product or inverse computes beyond rounding.
    dev = random_device(8, 64, 9, metal_frac=0.25, gap_offset=0.6)
    E = energy_grid(-1.5, 1.5, 10)
    T_o = o.transmission(dev, E, 1e-6)
    bar = MIXED_ABS
    base = None
    for tile_n in (64, 80, 96):
        for panel in (16, 32):
            (r,), _ = serve(rgf, [(dev, E, 1e-6)], slots=8, class_step=32,
                            tuning={64: {"slots": 8, "tile_n": tile_n, "panel": panel}})
            assert np.all(np.abs(r[0] - T_o) <= bar), (tile_n, panel)
            if base is None:
                base = r[0]
            assert np.abs(r[0] - base).max() <= 1e-10, (tile_n, panel)
    with rgf.Server(slots=8) as sv:
        with pytest.raises(rgf.RGFError) as ex:
            rgf.rgf_server_set_class(sv.handle, 64, 8, 72, 0)
        assert ex.value.status == rgf.RGF_E_INVALID
        sv.poll(sv.submit(dev, E[:2], 1e-6), timeout_us=300_000_000)
        with pytest.raises(rgf.RGFError) as ex:
            rgf.rgf_server_set_class(sv.handle, 64, 8, 64, 0)
        assert ex.value.status == rgf.RGF_E_STATE
