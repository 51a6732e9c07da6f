"""Host logic of the tile-shape autotuner (no GPU): every (units, blocks per
SM) pair is timed (and, for encode with at most two alphabets, 8 units with
the pair tables at each blocks-per-SM value), the fastest is chosen and stored
with its axes, a second call is served from the cache file, retune measures
again, and a damaged cache file is treated as empty."""
import json

import torch

from paper_1910_05109_gb300 import autotune


def fake_env(monkeypatch, timings):
    calls = []

    def time_units(op, src, src_off, dst, dst_off, alphabets, alph_id, units, workspace, reps=5):
        calls.append(units)
        return timings(units & 0xFF, (units >> 8) & 0xFF) + (0.01 if units >> 16 else 0.0)

    monkeypatch.setattr(autotune, "time_units", time_units)
    monkeypatch.setattr(autotune, "key", lambda op, n, total, device=None: f"gpu|{op}|{n}|{total}")
    return calls


def args(n=8, each=100):
    off = torch.arange(n + 1, dtype=torch.int64) * each
    src = torch.zeros(n * each, dtype=torch.uint8)
    return "encode", src, off, None, None, [None]


def grid(best_u, best_b):
    """A timing surface whose minimum is at (best_u, best_b)."""
    return lambda u, b: 0.1 + abs(u - best_u) + 0.5 * abs(b - best_b)


def test_searches_both_axes_then_caches(monkeypatch, tmp_path):
    calls = fake_env(monkeypatch, grid(4, 2))
    path = str(tmp_path / "tune.json")
    tile, t = autotune.best_units(*args(), path=path)
    assert tile == 4 | (2 << 8)
    assert autotune.describe(tile) == {"units": 4, "blocks_per_sm": 2, "pairs": False}
    assert sorted(t) == sorted(autotune.ENCODE_CHOICES) and len(calls) == 12
    assert {c & 0xFF for c in calls} == {2, 4, 8} and {(c >> 8) & 0xFF for c in calls} == {0, 1, 2}
    assert sorted(c for c in calls if c >> 16) == [8 | (b << 8) | (1 << 16) for b in (0, 1, 2)]
    stored = json.load(open(path))["gpu|encode|8|800"]
    assert stored["tile_units"] == tile and stored["units"] == 4 and stored["blocks_per_sm"] == 2
    assert len(stored["ms"]) == 12
    tile2, t2 = autotune.best_units(*args(), path=path)
    assert tile2 == tile and t2 == {} and len(calls) == 12  # cache hit: nothing timed


def test_pair_tables_chosen_when_fastest_and_only_for_encode(monkeypatch, tmp_path):
    calls = fake_env(monkeypatch, lambda u, b: 1.0)
    monkeypatch.setattr(autotune, "time_units",
                        lambda *a, **k: calls.append(a[7]) or (0.5 if a[7] >> 16 and
                                                               (a[7] >> 8) & 0xFF == 2 else 1.0))
    path = str(tmp_path / "tune.json")
    tile, _ = autotune.best_units(*args(), path=path)
    assert tile == 8 | (2 << 8) | (1 << 16)
    assert autotune.describe(tile) == {"units": 8, "blocks_per_sm": 2, "pairs": True}
    assert json.load(open(path))["gpu|encode|8|800"]["pairs"] is True
    calls.clear()
    autotune.best_units("decode", *args()[1:], path=path)
    assert len(calls) == 9 and not any(c >> 16 for c in calls)       # decode: no pair tables
    calls.clear()
    autotune.best_units("encode", *args(n=4)[1:5], [None, None, None], path=path)
    assert len(calls) == 9 and not any(c >> 16 for c in calls)       # three alphabets: none


def test_retune_and_other_keys(monkeypatch, tmp_path):
    path = str(tmp_path / "tune.json")
    fake_env(monkeypatch, grid(2, 0))
    assert autotune.best_units(*args(), path=path)[0] == 2
    calls = fake_env(monkeypatch, grid(8, 1))
    assert autotune.best_units(*args(), path=path)[0] == 2              # cached
    assert autotune.best_units(*args(), path=path, retune=True)[0] == 8 | (1 << 8)
    assert autotune.best_units(*args(n=16), path=path)[0] == 8 | (1 << 8)   # another batch size
    assert len(json.load(open(path))) == 2 and len(calls) == 24


def test_damaged_cache_file(monkeypatch, tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    fake_env(monkeypatch, grid(8, 0))
    assert autotune.best_units(*args(), path=str(path))[0] == 8
    assert json.load(open(path))["gpu|encode|8|800"]["tile_units"] == 8
