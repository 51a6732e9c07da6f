"""Serving: a continuous-batching request engine around the codec.

`Server` wraps the native engine (b64_server_* in the C ABI): it owns a
device arena of the memory budget and a pinned staging area, admits queued
requests whenever one of its streams is idle and arena space is free, and
runs each group as one batched launch (copy in, batched kernels, copy out),
overlapping groups on different streams.

`poisson_requests` builds the synthetic request stream (Poisson arrivals,
mixed encode/decode, lognormal sizes) and `run_open_loop` replays it in real
time: every request is submitted at its arrival time and its latency is
measured from that arrival to the poll that hands its result back.
"""
from __future__ import annotations

import collections
import ctypes
import time

import numpy as np

from . import binding as b64
from . import workloads as wl

COMPLETION = np.dtype([("tag", np.uint64), ("result", np.int64), ("latency_us", np.float64)])


class Server:
    def __init__(self, budget_bytes: int, alphabets, n_streams: int = 4,
                 max_batch_bytes: int = 0):
        self.alphabets = list(alphabets)
        arr = (ctypes.c_void_p * len(self.alphabets))(*[a.handle for a in self.alphabets])
        self.handle = b64.lib().b64_server_create(budget_bytes, n_streams, max_batch_bytes, arr,
                                                  len(self.alphabets))
        if not self.handle:
            raise b64.B64Error(b64.last_error())
        self._buf = np.zeros(1 << 16, COMPLETION)

    def submit(self, tag: int, op: int, alph_id: int, in_ptr: int, length: int, out_ptr: int,
               out_cap: int) -> None:
        rc = b64.lib().b64_server_submit(self.handle, tag, op, alph_id, in_ptr, length, out_ptr,
                                         out_cap)
        if rc != b64.B64_SUCCESS:
            raise b64.B64Error(b64.last_error())

    def submit_many(self, tags, ops, alph_ids, in_ptrs, lens, out_ptrs, out_caps) -> None:
        """Queues len(tags) requests in one call (b64_server_submit_many);
        pointers are host addresses as integers."""
        arrs = [np.ascontiguousarray(a, dtype=t) for a, t in (
            (tags, np.uint64), (ops, np.int32), (alph_ids, np.int32), (in_ptrs, np.uint64),
            (lens, np.uint64), (out_ptrs, np.uint64), (out_caps, np.uint64))]
        n = arrs[0].size
        for a in arrs[1:]:
            if a.size != n:
                raise ValueError("submit_many: arrays of different lengths")
        rc = b64.lib().b64_server_submit_many(self.handle, n, *[a.ctypes.data for a in arrs])
        if rc != n:
            raise b64.B64Error(b64.last_error())

    def poll(self) -> np.ndarray:
        n = b64.lib().b64_server_poll(self.handle, self._buf.ctypes.data, self._buf.size)
        if n < 0:
            raise b64.B64Error(b64.last_error())
        return self._buf[:n].copy()

    def outstanding(self) -> int:
        return b64.lib().b64_server_outstanding(self.handle)

    def batches(self) -> int:
        return int(b64.lib().b64_server_batches(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            b64.lib().b64_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


def poisson_requests(rate_hz: float, duration_s: float, seed_arrivals: int, seed_sizes: int,
                     decode_frac: float = 0.6, mu: float = 10.62, sigma: float = 2.0,
                     lo: int = 100, hi: int = 16 << 20, max_requests: int | None = None):
    """Arrival times, ops (1 = decode), sizes (input bytes; decode sizes are
    multiples of 4) and payload offsets into the pools."""
    t = wl.poisson_arrivals(rate_hz, duration_s, seed_arrivals)
    if max_requests is not None:
        t = t[:max_requests]
    n = t.size
    g = wl.rng(seed_sizes)
    ops = (g.random(n) < decode_frac).astype(np.int32)
    sizes = np.clip(np.rint(g.lognormal(mu, sigma, n)), lo, hi).astype(np.int64)
    sizes = np.where(ops == 1, np.maximum(sizes // 4 * 4, 4), sizes)
    pick = g.random(n)
    return t, ops, sizes, pick


class HostRing:
    """Output slots in one host buffer, released in submission order."""

    def __init__(self, nbytes: int):
        self.buf = np.ones(nbytes, np.uint8)        # touched up front
        self.cap = nbytes
        self.live = collections.deque()            # [offset, size, done]
        self.by_tag = {}

    def take(self, tag: int, size: int) -> int | None:
        size = (size + 63) // 64 * 64
        if not self.live:
            at = 0
        else:
            first = self.live[0][0]
            end = self.live[-1][0] + self.live[-1][1]
            # wrapped when the newest slot starts before the oldest; its end
            # may then equal the oldest slot's start (no room left)
            if self.live[-1][0] >= first:
                at = end if end + size <= self.cap else (0 if size <= first else None)
            else:
                at = end if end + size <= first else None
        if at is None or size > self.cap:
            return None
        slot = [at, size, False]
        self.live.append(slot)
        self.by_tag[tag] = slot
        return at

    def release(self, tag: int):
        self.by_tag.pop(tag)[2] = True
        while self.live and self.live[0][2]:
            self.live.popleft()


def run_open_loop(server: Server, arrivals, ops, sizes, pick, pools, out_bytes: int,
                  keep_outputs: bool = False):
    """Replays the request stream in real time. pools[op] = (host array, unit)
    where payloads are cut at random multiples of `unit`. Each pass hands every
    request that has arrived to the engine in one call (as many as the host
    output ring has room for, in one ring slot) and polls once. Returns
    per-request latency (s, arrival -> hand-back), results, and wall time.
    (Up to four arrivals go in one b64_server_submit call each, more in one
    b64_server_submit_many call.)"""
    n = arrivals.size
    lat = np.full(n, np.nan)
    results = np.zeros(n, np.int64)
    outputs = {} if keep_outputs else None
    ring = HostRing(out_bytes)
    ring_base = int(ring.buf.ctypes.data)
    caps = np.where(ops == 0, (sizes + 2) // 3 * 4, (sizes + 3) // 4 * 3).astype(np.int64)
    slots = (caps + 63) // 64 * 64                # each request's share of its group's slot
    base = np.array([int(p.ctypes.data) for p, _ in pools], np.int64)
    unit = np.array([u for _, u in pools], np.int64)
    span = np.array([p.size for p, _ in pools], np.int64)
    room = (span[ops] - sizes) // unit[ops]
    in_ptr = base[ops] + (pick * room).astype(np.int64) * unit[ops]
    out_at = np.zeros(n, np.int64)                # offset of each request's output in the ring
    group = np.zeros(n, np.int64)
    left = []                                     # per group: requests not yet handed back
    tags_all = np.arange(n, dtype=np.int64)
    zeros = np.zeros(n, np.int32)
    nxt = 0
    done = 0
    t0 = time.perf_counter()
    while done < n:
        now = time.perf_counter() - t0
        hi = nxt
        if nxt < n and arrivals[nxt] <= now:
            hi = nxt + 1
            if hi < n and arrivals[hi] <= now:
                hi = int(np.searchsorted(arrivals, now, side="right"))
        if hi > nxt:
            k = hi - nxt
            if k <= 4:                                # a few: plain Python is cheaper
                size = int(slots[nxt:hi].sum())
                at = ring.take(len(left), size)
                if at is not None:
                    for i in range(nxt, hi):
                        out_at[i] = at
                        group[i] = len(left)
                        server.submit(i, int(ops[i]), 0, int(in_ptr[i]), int(sizes[i]),
                                      ring_base + at, int(caps[i]))
                        at += int(slots[i])
                    left.append(k)
                    nxt = hi
            else:
                cum = np.cumsum(slots[nxt:hi])
                at = ring.take(len(left), int(cum[k - 1]))
                while at is None and k > 1:           # fewer, if the ring has less room
                    k //= 2
                    at = ring.take(len(left), int(cum[k - 1]))
                if at is not None:                    # else: host output space full, poll first
                    sl = slice(nxt, nxt + k)
                    out_at[sl] = at + cum[:k] - slots[sl]
                    group[sl] = len(left)
                    left.append(k)
                    server.submit_many(tags_all[sl], ops[sl], zeros[sl], in_ptr[sl], sizes[sl],
                                       ring_base + out_at[sl], caps[sl])
                    nxt += k
        comp = server.poll()
        if comp.size:
            t_now = time.perf_counter() - t0
            tags = comp["tag"].astype(np.int64)
            lat[tags] = t_now - arrivals[tags]
            results[tags] = comp["result"]
            if keep_outputs:
                for tag, r in zip(tags.tolist(), comp["result"].tolist()):
                    at = int(out_at[tag])
                    outputs[tag] = ring.buf[at:at + max(r, 0)].copy()
            for g in group[tags].tolist():
                left[g] -= 1
                if left[g] == 0:
                    ring.release(g)
            done += comp.size
    wall = time.perf_counter() - t0
    return lat, results, wall, outputs
