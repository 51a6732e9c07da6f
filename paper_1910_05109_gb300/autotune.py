"""Autotuner for the batched kernels' tile shape.

Three axes, all passed to the kernels in `tile_units`:
- bytes per thread: a tile is 32 threads x U units, a unit being 12 input
  bytes (encode) or 16 characters (decode), U in {2, 4, 8};
- threads per batch: B resident blocks of 8 warps per SM (0 = as many as fit,
  1 or 2), i.e. how many warps the batch is spread over. Within a tile a
  string's units are coded 32 at a time, one a thread, so a string of L bytes
  meets up to min(32, ceil(L / 12)) threads at once and ceil(L / (32 * 12 * U))
  tiles;
- for encode with U = 8 and at most two alphabets, whether whole tiles go
  through 4096-entry character-pair tables (B64_TILE_PAIRS, bit 16): faster
  for long strings, slower where many strings share tiles.
The tuner times every choice on the caller's own batch with CUDA events,
keeps the fastest, and caches it in a JSON file keyed by GPU name, SM count,
operation and the batch's size buckets (log2 of the string count and of the
mean string length). The value returned (and cached) is U | B << 8, with
bit 16 for the pair tables.

The cache lives in $B64GPU_CACHE, else $XDG_CACHE_HOME/b64gpu/autotune.json,
else ~/.cache/b64gpu/autotune.json.
"""
from __future__ import annotations

import json
import math
import os
import threading

import torch

from . import binding as b64

UNITS = (2, 4, 8)
BLOCKS = (0, 1, 2)          # resident blocks an SM (0: as many as fit)
TILE_PAIRS = 1 << 16        # B64_TILE_PAIRS: encode's whole tiles through pair tables
CHOICES = tuple(u | (b << 8) for b in BLOCKS for u in UNITS)
# encode with 8 units also tries the pair tables (batches of at most 2 alphabets)
ENCODE_CHOICES = CHOICES + tuple(8 | (b << 8) | TILE_PAIRS for b in BLOCKS)


def choices(op: str, n_alphabets: int) -> tuple:
    """The tile_units values the tuner times for op."""
    return ENCODE_CHOICES if op == "encode" and n_alphabets <= 2 else CHOICES


def describe(tile: int) -> dict:
    """The axes of a tile_units value."""
    return {"units": tile & 0xFF, "blocks_per_sm": (tile >> 8) & 0xFF,
            "pairs": bool(tile & TILE_PAIRS)}
_lock = threading.Lock()


def cache_path() -> str:
    if os.environ.get("B64GPU_CACHE"):
        return os.environ["B64GPU_CACHE"]
    base = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(base, "b64gpu", "autotune.json")


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path: str, table: dict) -> None:
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def key(op: str, n: int, total_bytes: int, device=None) -> str:
    props = torch.cuda.get_device_properties(device or torch.cuda.current_device())
    mean = total_bytes / max(n, 1)
    nb = int(math.log2(max(n, 1)))
    lb = int(math.log2(max(mean, 1)))
    return f"{props.name}|sm{props.multi_processor_count}|{op}|n2^{nb}|len2^{lb}"


def time_units(op: str, src, src_off, dst, dst_off, alphabets, alph_id, units: int,
               workspace, reps: int = 5) -> float:
    """Median milliseconds of one batched call with tile size `units`."""
    fn = b64.encode_batch if op == "encode" else b64.decode_batch
    stream = torch.cuda.current_stream()
    for _ in range(2):
        fn(src, src_off, dst, dst_off, alphabets, alph_id, None, units, workspace)
    times = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn(src, src_off, dst, dst_off, alphabets, alph_id, None, units, workspace)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    times.sort()
    return times[len(times) // 2]


def best_units(op: str, src, src_off, dst, dst_off, alphabets, alph_id=None,
               path: str | None = None, retune: bool = False) -> tuple[int, dict]:
    """The tile shape for this batch: from the cache, else measured and
    stored. Returns (tile_units, {tile_units: ms} measured now, or {} on a
    cache hit)."""
    path = path or cache_path()
    n = src_off.numel() - 1
    total = int(src_off[-1].item() - src_off[0].item())
    k = key(op, n, total, src.device)
    with _lock:
        table = _load(path)
        if not retune and k in table:
            return int(table[k]["tile_units"]), {}
    ws = b64.batch_workspace(n, src.device)
    timings = {u: time_units(op, src, src_off, dst, dst_off, alphabets, alph_id, u, ws)
               for u in choices(op, len(alphabets))}
    best = min(timings, key=timings.get)
    with _lock:
        table = _load(path)
        table[k] = {"tile_units": best, **describe(best),
                    "ms": {str(u): t for u, t in timings.items()}}
        _store(path, table)
    return best, timings
