"""The batched decode that allocates nothing (b64_decode_batch_noalloc).

It exists for callers that cannot allocate device memory where they decode
(a plugin given only its buffers, a process whose memory budget belongs to
someone else, a path that must not enter an allocator): its workspace is a
file-scope device array of the library. These tests call it through the C ABI
and check that it returns exactly what the oracle and b64_decode_batch (with a
caller workspace) return, on two different batches in a row, so a second call
cannot see what the first left in the shared array; that a batch of exactly
the array's limit of strings decodes correctly; that a call after the first
leaves the device's free memory unchanged; and that a batch over the limit is
refused with a clear message.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1910_05109_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

LIMIT = 65536


@pytest.fixture(scope="module")
def b64():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import __graft_entry__
    __graft_entry__.build()
    from paper_1910_05109_gb300 import binding
    binding.lib()
    return binding


def encoded_batch(orc, count, seed, error_rate):
    lengths = wl.lognormal_lengths(count, seed, 700, 1.4, 1, 1 << 15)
    lengths[:4] = [0, 1, 2, 3]
    off = wl.offsets_from_lengths(lengths)
    data = wl.random_bytes(int(off[-1]), seed + 1)
    aid = wl.bernoulli(count, seed + 2).astype(np.uint8)
    padded = (aid == 0).astype(np.int32)
    elen = np.array([orc.encoded_length(int(off[i + 1] - off[i]), bool(padded[i]))
                     for i in range(count)], np.int64)
    eoff = wl.offsets_from_lengths(elen)
    text, _ = orc.encode_batch(data, off, eoff, orc.standard_alphabet() + orc.url_alphabet(),
                               aid.astype(np.int32), padded, int(eoff[-1]))
    text = text.copy()
    g = wl.rng(seed + 3)
    for i in np.nonzero(g.random(count) < error_rate)[0]:
        m = int(eoff[i + 1] - eoff[i])
        if m:
            text[eoff[i] + int(g.integers(0, m))] = 0xFF
    return text, eoff, aid


def oracle_decode(orc, text, eoff, aid):
    """The oracle's results and decoded bytes, at b64_batch_offsets' layout
    (capacity 3 * ceil(len / 4) per string)."""
    lens = eoff[1:] - eoff[:-1]
    doff = wl.offsets_from_lengths((lens + 3) // 4 * 3)
    padded = (aid == 0).astype(np.int32)
    dst, res = orc.decode_batch(text, eoff, doff, orc.standard_alphabet() + orc.url_alphabet(),
                                aid.astype(np.int32), padded, int(doff[-1]))
    return res, dst, doff


def check_against_oracle(orc, text, eoff, aid, got_res, got_dst):
    want_res, want_dst, doff = oracle_decode(orc, text, eoff, aid)
    res = got_res.cpu().numpy()
    assert np.array_equal(res, want_res)
    out = got_dst.cpu().numpy()
    for i in np.nonzero(res > 0)[0]:
        o = int(doff[i])
        assert np.array_equal(out[o:o + res[i]], want_dst[o:o + res[i]]), i


def run_both(b64, text, eoff, aid, units):
    alphs = [b64.Alphabet.standard(), b64.Alphabet.url()]
    src = torch.from_numpy(text).cuda()
    off = torch.from_numpy(eoff).cuda()
    d_aid = torch.from_numpy(aid).cuda()
    n = eoff.size - 1
    dst_off = b64.batch_offsets(off, alphs, d_aid, decode=True)
    cap = int(dst_off[-1]) + 64
    want_dst = torch.full((cap,), 0xA5, dtype=torch.uint8, device="cuda")
    want_res = b64.decode_batch(src, off, want_dst, dst_off, alphs, d_aid, tile_units=units)
    got_dst = torch.full((cap,), 0xA5, dtype=torch.uint8, device="cuda")
    got_res = torch.full((n,), 7, dtype=torch.int64, device="cuda")
    arr = (ctypes.c_void_p * 2)(alphs[0].handle, alphs[1].handle)
    rc = b64.lib().b64_decode_batch_noalloc(
        src.data_ptr(), off.data_ptr(), n, got_dst.data_ptr(), dst_off.data_ptr(), arr, 2,
        d_aid.data_ptr(), got_res.data_ptr(), units, torch.cuda.current_stream().cuda_stream)
    assert rc == b64.B64_SUCCESS, b64.last_error()
    torch.cuda.synchronize()
    return want_res, got_res, want_dst, got_dst


def test_noalloc_equals_workspace_call_twice_in_a_row(b64, orc):
    first = encoded_batch(orc, 3000, seed=61, error_rate=0.2)    # many per-string errors
    second = encoded_batch(orc, 2500, seed=62, error_rate=0.0)   # none: stale words would show
    for (text, eoff, aid), units in ((first, 4), (second, 2)):
        want_res, got_res, want_dst, got_dst = run_both(b64, text, eoff, aid, units)
        assert torch.equal(got_res, want_res)
        assert torch.equal(got_dst, want_dst)
        check_against_oracle(orc, text, eoff, aid, got_res, got_dst)
    assert int((want_res < 0).sum()) == 0


def test_noalloc_at_its_limit_and_without_new_device_memory(b64, orc):
    """Exactly 65,536 strings (the largest batch it accepts), decoded
    twice: both calls give the oracle's results, and the second call, made
    once every buffer exists and the first call has loaded the kernels,
    leaves the device's free memory as it was."""
    text, eoff, aid = encoded_batch(orc, LIMIT, seed=63, error_rate=0.05)
    alphs = [b64.Alphabet.standard(), b64.Alphabet.url()]
    src = torch.from_numpy(text).cuda()
    off = torch.from_numpy(eoff).cuda()
    d_aid = torch.from_numpy(aid).cuda()
    dst_off = b64.batch_offsets(off, alphs, d_aid, decode=True)
    dst = torch.zeros(int(dst_off[-1]) + 64, dtype=torch.uint8, device="cuda")
    res = torch.zeros(LIMIT, dtype=torch.int64, device="cuda")
    arr = (ctypes.c_void_p * 2)(alphs[0].handle, alphs[1].handle)
    stream = torch.cuda.current_stream().cuda_stream

    def call():
        rc = b64.lib().b64_decode_batch_noalloc(
            src.data_ptr(), off.data_ptr(), LIMIT, dst.data_ptr(), dst_off.data_ptr(), arr, 2,
            d_aid.data_ptr(), res.data_ptr(), 0, stream)
        assert rc == b64.B64_SUCCESS, b64.last_error()
        torch.cuda.synchronize()

    call()
    check_against_oracle(orc, text, eoff, aid, res, dst)
    res.fill_(7)
    dst.fill_(0)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    call()
    assert torch.cuda.mem_get_info()[0] == free_before
    check_against_oracle(orc, text, eoff, aid, res, dst)
    assert int((res < 0).sum()) > 0


def test_noalloc_refuses_batches_over_its_limit(b64):
    n = LIMIT + 1
    off = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    res = torch.zeros(n, dtype=torch.int64, device="cuda")
    buf = torch.zeros(16, dtype=torch.uint8, device="cuda")
    arr = (ctypes.c_void_p * 1)(b64.Alphabet.standard().handle)
    rc = b64.lib().b64_decode_batch_noalloc(buf.data_ptr(), off.data_ptr(), n, buf.data_ptr(),
                                            off.data_ptr(), arr, 1, None, res.data_ptr(), 0, None)
    assert rc == b64.B64_ERR_INVALID_ARGUMENT
    assert "65536" in b64.last_error() and "limit" in b64.last_error()
