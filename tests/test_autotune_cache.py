"""Host logic of the tile-size autotuner (no GPU): the fastest tile size is
chosen and stored, a second call is served from the cache file, retune
measures again, and a damaged cache file is treated as empty."""
import json

import torch

from paper_1910_05109_gb300 import autotune


def fake_env(monkeypatch, timings):
    calls = []

    def time_units(op, src, src_off, dst, dst_off, alphabets, alph_id, units, workspace, reps=5):
        calls.append(units)
        return timings[units]

    monkeypatch.setattr(autotune, "time_units", time_units)
    monkeypatch.setattr(autotune, "key", lambda op, n, total, device=None: f"gpu|{op}|{n}|{total}")
    return calls


def args(n=8, each=100):
    off = torch.arange(n + 1, dtype=torch.int64) * each
    src = torch.zeros(n * each, dtype=torch.uint8)
    return "encode", src, off, None, None, [None]


def test_measures_then_caches(monkeypatch, tmp_path):
    calls = fake_env(monkeypatch, {1: 0.9, 2: 0.5, 4: 0.3, 8: 0.4})
    path = str(tmp_path / "tune.json")
    units, t = autotune.best_units(*args(), path=path)
    assert units == 4 and sorted(t) == [1, 2, 4, 8] and calls == [1, 2, 4, 8]
    stored = json.load(open(path))
    assert stored["gpu|encode|8|800"]["units"] == 4
    units, t = autotune.best_units(*args(), path=path)
    assert units == 4 and t == {} and calls == [1, 2, 4, 8]  # cache hit: nothing timed


def test_retune_and_other_keys(monkeypatch, tmp_path):
    path = str(tmp_path / "tune.json")
    fake_env(monkeypatch, {1: 0.9, 2: 0.2, 4: 0.3, 8: 0.4})
    assert autotune.best_units(*args(), path=path)[0] == 2
    calls = fake_env(monkeypatch, {1: 0.1, 2: 0.2, 4: 0.3, 8: 0.4})
    assert autotune.best_units(*args(), path=path)[0] == 2           # cached
    assert autotune.best_units(*args(), path=path, retune=True)[0] == 1
    assert autotune.best_units(*args(n=16), path=path)[0] == 1       # another batch size
    assert len(json.load(open(path))) == 2 and len(calls) == 8


def test_damaged_cache_file(monkeypatch, tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    fake_env(monkeypatch, {1: 0.4, 2: 0.3, 4: 0.2, 8: 0.1})
    assert autotune.best_units(*args(), path=str(path))[0] == 8
    assert json.load(open(path))["gpu|encode|8|800"]["units"] == 8
