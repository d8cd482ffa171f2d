"""Host logic of the autotuner (no GPU): the coordinate search and the table
format that the server loads."""
import json

from paper_2609_37058_b300 import autotune, rgf


def test_coordinate_search_finds_the_best_on_each_axis():
    # A separable figure of merit with its optimum at (64, 16, 296).
    score = {"tile_n": {96: 1.0, 80: 1.5, 64: 2.0}, "panel": {32: 1.0, 16: 1.2}, "slots": {148: 1.0, 74: 0.7, 296: 1.1, 592: 1.05}}
    calls = []

    def measure(bc, cfg):
        calls.append(cfg)
        return score["tile_n"][cfg["tile_n"]] * score["panel"][cfg["panel"]] * score["slots"][cfg["slots"]]

    cfg, rate, log = autotune.search(measure, 128)
    assert cfg == {"tile_n": 64, "panel": 16, "slots": 296}
    assert abs(rate - 2.0 * 1.2 * 1.1) < 1e-12
    # start, two tiles, one panel, two slot counts, then one doubling that does not pay
    assert len(calls) == len(log) == 1 + 2 + 1 + 2 + 1
    assert all(set(c) == {"tile_n", "panel", "slots"} for c in calls)


def test_search_keeps_the_start_when_nothing_is_faster():
    # Equal rates: start tile and panel, and the fewest slots (least memory).
    cfg, rate, _ = autotune.search(lambda bc, c: 1.0, 64)
    assert cfg == {"tile_n": autotune.TILES[0], "panel": autotune.PANELS[0], "slots": min(autotune.SLOTS)}


def test_tuning_table_round_trip(tmp_path):
    p = tmp_path / "t.json"
    p.write_text(json.dumps({"device": "x", "classes": {"256": {"slots": 148, "tile_n": 64, "panel": 32,
                                                                  "energy_points_per_s": 10.0}}}))
    t = rgf.load_tuning(str(p))
    assert t == {256: {"slots": 148, "tile_n": 64, "panel": 32, "energy_points_per_s": 10.0}}
    assert rgf.load_tuning(str(tmp_path / "missing.json")) == {}


def test_slot_doubling_stops_at_the_cap():
    cfg, rate, log = autotune.search(lambda bc, c: float(c["slots"]), 64)
    assert cfg["slots"] == autotune.MAX_SLOTS
    assert max(c["slots"] for c in log) == autotune.MAX_SLOTS


def test_smallest_slot_count_within_tolerance_is_kept():
    rates = {74: 0.8, 148: 1.0, 296: 1.10, 592: 1.14, 1184: 1.16}
    cfg, rate, _ = autotune.search(lambda bc, c: rates[c["slots"]], 256)
    assert cfg["slots"] == 592 and rate == 1.14  # 1.14 >= 0.97 * 1.16


def test_tune_cache_environment_variable(tmp_path, monkeypatch):
    p = tmp_path / "mine.json"
    p.write_text(json.dumps({"classes": {"96": {"slots": 296, "tile_n": 80, "panel": 16}}}))
    monkeypatch.setenv("RGF_TUNE_CACHE", str(p))
    assert rgf.tuning_path() == str(p)
    assert rgf.load_tuning() == {96: {"slots": 296, "tile_n": 80, "panel": 16}}
    monkeypatch.delenv("RGF_TUNE_CACHE")
    assert rgf.tuning_path() == rgf.TUNING_PATH
