"""Serving engine: continuous batching under a device-memory budget.

Requests arrive as a Poisson stream (mixed encode / decode, lognormal sizes)
and are replayed in real time. Every result, length and bytes, must equal the
oracle's and the same request served alone. The decode payloads carry seeded
invalid bytes, so per-request error offsets pass through the engine too. One
run uses the serving workload's full size range (up to 16 MiB) under a small
budget, so large requests wait for memory and the arena ring wraps; a small
budget forces waits; a request larger than the budget is refused.
"""
import base64

import numpy as np
import pytest
import torch

from paper_1910_05109_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def with_bad_bytes(text: np.ndarray, every: int, seed: int) -> np.ndarray:
    """A copy of `text` with one 0xFF at a seeded position in about every
    `every` bytes (none in the last 8 bytes)."""
    out = text.copy()
    g = wl.rng(seed)
    k = max(1, text.size // every)
    out[g.integers(0, text.size - 8, k)] = 0xFF
    return out


@pytest.fixture(scope="module")
def env(orc):
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import __graft_entry__
    __graft_entry__.build()
    from paper_1910_05109_gb300 import binding, serve
    raw = wl.random_bytes(8 << 20, 5)
    text = with_bad_bytes(orc.encode(raw), 256 << 10, 15)   # decode payloads
    return binding, serve, [(raw, 1), (text, 4)]


class Alone:
    """One engine that serves one request at a time (nothing else in flight)."""

    def __init__(self, serve, b64, budget):
        self.srv = serve.Server(budget, [b64.Alphabet.standard()], n_streams=1)

    def run(self, op, data):
        cap = (data.size + 2) // 3 * 4 if op == 0 else (data.size + 3) // 4 * 3
        out = np.zeros(max(cap, 1), np.uint8)
        self.srv.submit(7, op, 0, data.ctypes.data, data.size, out.ctypes.data, cap)
        while True:
            c = self.srv.poll()
            if c.size:
                r = int(c["result"][0])
                return r, out[:max(r, 0)].copy()

    def close(self):
        self.srv.close()


def payloads(ops, sizes, pick, pools):
    out = []
    for i in range(ops.size):
        arr, unit = pools[ops[i]]
        room = (arr.size - sizes[i]) // unit
        off = int(pick[i] * room) * unit
        out.append((int(ops[i]), arr[off:off + sizes[i]]))
    return out


def check_every_result(orc, reqs, results, outputs, alone=None):
    """Every request's result and bytes against the oracle, and (if given)
    against the same request served alone. Returns the number of decode
    requests that reported an error."""
    errors = 0
    for i, (op, data) in enumerate(reqs):
        if op == 0:
            want = orc.encode(data)
            want_r = want.size
        else:
            want_r, want = orc.decode(data)
            errors += want_r < 0
        assert results[i] == want_r, (i, op, data.size, results[i], want_r)
        if want_r >= 0:
            assert np.array_equal(outputs[i], want), i
        if alone is not None:
            r, out = alone.run(op, data)
            assert r == results[i] and np.array_equal(out, outputs[i][:max(r, 0)]), i
    return errors


def test_mix_equals_alone_and_oracle(env, orc):
    b64, serve, pools = env
    arrivals, ops, sizes, pick = serve.poisson_requests(20_000, 0.25, 4, 5, hi=1 << 18)
    srv = serve.Server(256 << 20, [b64.Alphabet.standard()], n_streams=4)
    lat, results, wall, outputs = serve.run_open_loop(srv, arrivals, ops, sizes, pick, pools,
                                                      1 << 30, keep_outputs=True)
    n = arrivals.size
    assert n > 3000 and not np.isnan(lat).any()
    assert srv.batches() < n                    # requests were batched together
    srv.close()
    alone = Alone(serve, b64, 64 << 20)
    errors = check_every_result(orc, payloads(ops, sizes, pick, pools), results, outputs, alone)
    alone.close()
    assert 50 < errors < int((ops == 1).sum())   # some decode requests fail, most do not


def test_full_size_range_under_a_small_budget(env, orc):
    """The serving workload's size range (lognormal up to 16 MiB) through a
    48 MiB arena with an 8 MiB batch cap: requests larger than the cap run
    in batches of their own, large ones wait for arena space, the ring wraps.
    Every result is checked against the oracle and against a lone run."""
    b64, serve, _ = env
    raw = wl.random_bytes(48 << 20, 25)
    text = with_bad_bytes(orc.encode(raw), 4 << 20, 26)
    pools = [(raw, 1), (text, 4)]
    arrivals, ops, sizes, pick = serve.poisson_requests(400, 2.0, 27, 54)
    assert (sizes == 16 << 20).sum() == 4 and (sizes > 4 << 20).sum() == 11  # at the clip
    srv = serve.Server(48 << 20, [b64.Alphabet.standard()], n_streams=4,
                       max_batch_bytes=8 << 20)
    lat, results, wall, outputs = serve.run_open_loop(srv, arrivals, ops, sizes, pick, pools,
                                                      2 << 30, keep_outputs=True)
    assert not np.isnan(lat).any()
    batches = srv.batches()
    srv.close()
    assert batches > 1
    alone = Alone(serve, b64, 48 << 20)
    errors = check_every_result(orc, payloads(ops, sizes, pick, pools), results, outputs, alone)
    alone.close()
    assert errors > 0


def test_small_budget_waits_and_refuses(env, orc):
    b64, serve, pools = env
    arrivals, ops, sizes, pick = serve.poisson_requests(20_000, 0.05, 6, 7, hi=1 << 18)
    srv = serve.Server(4 << 20, [b64.Alphabet.standard()], n_streams=2)
    lat, results, wall, outputs = serve.run_open_loop(srv, arrivals, ops, sizes, pick, pools,
                                                      1 << 28, keep_outputs=True)
    check_every_result(orc, payloads(ops, sizes, pick, pools), results, outputs)
    big = np.zeros(8 << 20, np.uint8)
    out = np.zeros((8 << 20) // 3 * 4 + 4, np.uint8)
    with pytest.raises(b64.B64Error, match="budget"):
        srv.submit(1, 0, 0, big.ctypes.data, big.size, out.ctypes.data, out.size)
    # the server holds one alphabet: id 1 is refused, not coded with another
    with pytest.raises(b64.B64Error, match="bad argument"):
        srv.submit(2, 0, 1, big.ctypes.data, 12, out.ctypes.data, 16)
    srv.close()


def test_burst_larger_than_budget_drains(env):
    """Requests queued all at once whose total is many times the budget (and
    a batch cap far above it) are split into batches that each fit the arena,
    and all of them complete."""
    import time
    b64, serve, pools = env
    raw, text = pools[0][0], pools[1][0]
    text = text[:text.size // 4 * 4]
    srv = serve.Server(2 << 20, [b64.Alphabet.standard()], n_streams=2,
                       max_batch_bytes=256 << 20)
    g = wl.rng(21)
    reqs, outs = [], []
    for i in range(600):
        op = int(g.integers(0, 2))
        size = int(g.integers(1, 40_000))
        if op == 1:
            size = size // 4 * 4 + 4
            off = int(g.integers(0, (text.size - size) // 4)) * 4
            data = text[off:off + size]
            cap = size // 4 * 3
        else:
            off = int(g.integers(0, raw.size - size))
            data = raw[off:off + size]
            cap = (size + 2) // 3 * 4
        out = np.zeros(cap, np.uint8)
        srv.submit(i, op, 0, data.ctypes.data, data.size, out.ctypes.data, cap)
        reqs.append((op, data))
        outs.append(out)
    results = {}
    deadline = time.monotonic() + 60
    while len(results) < len(reqs):
        assert time.monotonic() < deadline, f"{len(results)} of {len(reqs)} done"
        for c in srv.poll():
            results[int(c["tag"])] = int(c["result"])
    assert srv.batches() > 1
    for i, (op, data) in enumerate(reqs):
        if op == 0:
            want = base64.b64encode(data.tobytes())
            assert results[i] == len(want), i
            assert outs[i][:results[i]].tobytes() == want, i
        elif 0xFF in data:                       # the payloads carry seeded bad bytes
            assert results[i] == -(int(np.argmax(data == 0xFF)) + 1), i
        else:
            want = base64.b64decode(data.tobytes())
            assert results[i] == len(want), i
            assert outs[i][:results[i]].tobytes() == want, i
    srv.close()
