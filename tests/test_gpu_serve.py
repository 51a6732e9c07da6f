"""Serving engine: continuous batching under a device-memory budget.

Requests arrive as a Poisson stream (mixed encode / decode, lognormal sizes)
and are replayed in real time; every result must be identical to the same
request served alone, and the sampled ones must equal the oracle's. A small
budget forces requests to wait for memory; a request larger than the budget
is refused.
"""
import numpy as np
import pytest
import torch

from paper_1910_05109_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env(orc):
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import __graft_entry__
    __graft_entry__.build()
    from paper_1910_05109_gb300 import binding, serve
    raw = wl.random_bytes(8 << 20, 5)
    text = orc.encode(raw)                      # decode payloads: valid base64
    return binding, serve, [(raw, 1), (text, 4)]


def serve_alone(serve, b64, req, pools):
    op, data = req
    srv = serve.Server(64 << 20, [b64.Alphabet.standard()], n_streams=1)
    cap = (data.size + 2) // 3 * 4 if op == 0 else (data.size + 3) // 4 * 3
    out = np.zeros(max(cap, 1), np.uint8)
    srv.submit(7, op, 0, data.ctypes.data, data.size, out.ctypes.data, cap)
    while True:
        c = srv.poll()
        if c.size:
            r = int(c["result"][0])
            srv.close()
            return r, out[:max(r, 0)].copy()


def payloads(ops, sizes, pick, pools):
    out = []
    for i in range(ops.size):
        arr, unit = pools[ops[i]]
        room = (arr.size - sizes[i]) // unit
        off = int(pick[i] * room) * unit
        out.append((int(ops[i]), arr[off:off + sizes[i]]))
    return out


def test_mix_equals_alone_and_oracle(env, orc):
    b64, serve, pools = env
    arrivals, ops, sizes, pick = serve.poisson_requests(20_000, 0.25, 4, 5, hi=1 << 18)
    srv = serve.Server(256 << 20, [b64.Alphabet.standard()], n_streams=4)
    lat, results, wall, outputs = serve.run_open_loop(srv, arrivals, ops, sizes, pick, pools,
                                                      1 << 30, keep_outputs=True)
    n = arrivals.size
    assert n > 3000 and not np.isnan(lat).any()
    assert srv.batches() < n                    # requests were batched together
    reqs = payloads(ops, sizes, pick, pools)
    for i in range(n):
        op, data = reqs[i]
        want_len = (data.size + 2) // 3 * 4 if op == 0 else data.size // 4 * 3 - \
            int((data[-2:] == ord("=")).sum())
        assert results[i] == want_len, i
    g = wl.rng(9)
    for i in g.choice(n, 150, replace=False):
        r, out = serve_alone(serve, b64, reqs[i], pools)
        assert r == results[i] and np.array_equal(out, outputs[i]), i
        op, data = reqs[i]
        want = orc.encode(data) if op == 0 else orc.decode(data)[1]
        assert np.array_equal(outputs[i], want), i
    srv.close()


def test_small_budget_waits_and_refuses(env):
    b64, serve, pools = env
    arrivals, ops, sizes, pick = serve.poisson_requests(20_000, 0.05, 6, 7, hi=1 << 18)
    srv = serve.Server(4 << 20, [b64.Alphabet.standard()], n_streams=2)
    lat, results, wall, outputs = serve.run_open_loop(srv, arrivals, ops, sizes, pick, pools,
                                                      1 << 28, keep_outputs=True)
    reqs = payloads(ops, sizes, pick, pools)
    for i in range(arrivals.size):
        op, data = reqs[i]
        if op == 0:
            assert np.array_equal(outputs[i], np.frombuffer(
                __import__("base64").b64encode(data.tobytes()), np.uint8)), i
        else:
            assert results[i] >= 0, i
    big = np.zeros(8 << 20, np.uint8)
    out = np.zeros((8 << 20) // 3 * 4 + 4, np.uint8)
    with pytest.raises(b64.B64Error, match="budget"):
        srv.submit(1, 0, 0, big.ctypes.data, big.size, out.ctypes.data, out.size)
    srv.close()


def test_burst_larger_than_budget_drains(env):
    """Requests queued all at once whose total is many times the budget (and
    a batch cap far above it) are split into batches that each fit the arena,
    and all of them complete."""
    import base64
    import time
    b64, serve, pools = env
    raw, text = pools[0][0], pools[1][0]
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
        want = base64.b64encode(data.tobytes()) if op == 0 else base64.b64decode(data.tobytes())
        assert results[i] == len(want), i
        assert outs[i][:results[i]].tobytes() == want, i
    srv.close()
