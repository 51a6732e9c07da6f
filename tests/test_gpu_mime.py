"""Parity of the MIME (whitespace-skipping) strict decode with the oracle.

Inputs are base64 text from the oracle, line-wrapped with CRLF every 76
characters or with CR/LF/space inserted at random places (long runs that
cover whole tiles included), '=' padding split across tiles, injected bad
bytes, both padding modes, any alignment; the full-size case is 256 MiB of
seed-3 random bytes (357,913,944 characters, 367,332,730 bytes with CRLF),
plus 256 documents of 1 MiB each with a stray bad byte at p = 0.01.
"""
import numpy as np
import pytest
import torch

from paper_1910_05109_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TILE = 4096  # raw bytes per segment of the decode kernel


@pytest.fixture(scope="module")
def b64():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import __graft_entry__
    __graft_entry__.build()
    from paper_1910_05109_gb300 import binding
    binding.lib()
    yield binding
    assert binding.device_fault_flag() == 0


def run(b64, text, alph, src_off=0, dst_off=0, strict_tail=False):
    """Decodes text; canary bytes around dst must survive: past the result
    for inputs whose line layout holds throughout (strict_tail), past
    b64_decoded_max_length otherwise (the one-pass kernel may have written
    segments after a layout break at their layout offsets)."""
    buf = torch.empty(text.size + src_off + 16, dtype=torch.uint8, device="cuda")
    src = buf[src_off:src_off + text.size]
    if text.size:
        src.copy_(torch.from_numpy(np.ascontiguousarray(text)))
    cap = b64.decoded_max_length(text.size)
    out = torch.full((cap + dst_off + 32,), 0xA5, dtype=torch.uint8, device="cuda")
    r, _ = b64.mime_decode(src, alph, out[dst_off:dst_off + max(cap, 1)])
    host = out.cpu().numpy()
    assert (host[:dst_off] == 0xA5).all()
    written = r if r >= 0 and strict_tail else cap
    assert (host[dst_off + written:] == 0xA5).all()
    return r, host[dst_off:dst_off + max(r, 0)]


def check(b64, orc, text, alph, chars, padded, **kw):
    want_r, want = orc.decode(text, chars, padded, mime=True)
    r, got = run(b64, text, alph, **kw)
    assert r == want_r, (r, want_r)
    if r >= 0:
        assert np.array_equal(got, want)
    return r


def test_wrapped_sizes(b64, orc):
    std = b64.Alphabet.standard()
    for i, n in enumerate([0, 1, 2, 3, 56, 57, 58, 1000, 6144, 6145, 6146, 12287, 50_000,
                           200_001]):
        text = wl.mime_wrap(orc.encode(wl.random_bytes(n, 300 + i)))
        assert check(b64, orc, text, std, orc.standard_alphabet(), True, strict_tail=True) == n


def test_random_whitespace_and_long_runs(b64, orc):
    url = b64.Alphabet.url()
    for i in range(12):
        data = wl.random_bytes(int(wl.rng(i).integers(0, 60_000)), 400 + i)
        text = orc.encode(data, orc.url_alphabet(), False)
        text = wl.insert_spaces(text, seed=500 + i, count=int(text.size * 0.3) + 1)
        if i % 3 == 0:  # a run of spaces longer than a tile somewhere in the middle
            p = text.size // 2
            text = np.concatenate([text[:p], np.full(TILE * 2 + 5, 32, np.uint8), text[p:]])
        assert check(b64, orc, text, url, orc.url_alphabet(), False) == data.size


def test_padding_across_tile_edges(b64, orc):
    std = b64.Alphabet.standard()
    for n in (1, 2, 4, 5):
        body = orc.encode(wl.random_bytes(6141 + n, 600 + n))   # ends with '=' or '=='
        for gap in range(0, 6):
            # place the padding right at a tile boundary, with whitespace around it
            k = int((body[-2:] == ord("=")).sum())
            head, pad = body[:body.size - k], body[body.size - k:]
            filler = np.full((TILE - (head.size + gap) % TILE) % TILE, 10, np.uint8)
            text = np.concatenate([head, filler, np.full(gap, 13, np.uint8), pad,
                                   np.full(gap, 32, np.uint8)])
            check(b64, orc, text, std, orc.standard_alphabet(), True)


def test_errors_and_alignment(b64, orc):
    std = b64.Alphabet.standard()
    base = wl.mime_wrap(orc.encode(wl.random_bytes(40_000, 700)))
    g = wl.rng(701)
    for t in range(60):
        text = base.copy()
        p = int(g.integers(0, text.size))
        text[p] = int(g.choice([0x00, 0x09, 0x2D, 0x3D, 0x7F, 0xC3, 0xFF, ord("+")]))
        check(b64, orc, text, std, orc.standard_alphabet(), True, src_off=t % 7, dst_off=t % 5)
    for bad in (b"QQ\r\n=A", b"QQ=\r\n=", b"Q===", b"QQ==\r\nQQ==", b"QQ \t", b"\r\n\r\n",
                b"QUJD\r\n", b" QUI=\r\n", b"QQ\r\n"):
        check(b64, orc, np.frombuffer(bad, np.uint8), std, orc.standard_alphabet(), True)


def test_config4_full_size(b64, orc):
    """256 MiB of seed-3 random bytes, encoded and wrapped at 76 characters
    with CRLF (no trailing CRLF): 367,332,730 bytes of input."""
    data = wl.random_bytes(256 << 20, 3)
    text = wl.mime_wrap(orc.encode(data))
    assert text.size == 367_332_730
    src = torch.from_numpy(text).cuda()
    r, dec = b64.mime_decode(src, b64.Alphabet.standard())
    want_r, want = orc.decode(text, mime=True)
    assert r == want_r == data.size
    assert torch.equal(dec, torch.from_numpy(want).cuda())


def test_config4_documents_with_stray_bytes(b64, orc):
    """256 documents of 1 MiB source each; each gets a stray bad byte with
    p = 0.01 (seed 13, at least one forced); offsets against the oracle."""
    g = wl.rng(13)
    hit = g.random(256) < 0.01
    if not hit.any():
        hit[int(g.integers(0, 256))] = True
    std = b64.Alphabet.standard()
    ws = b64.mime_workspace(1_500_000)
    for d in range(256):
        text = wl.mime_wrap(orc.encode(wl.random_bytes(1 << 20, 10_000 + d)))
        if hit[d]:
            text[int(g.integers(0, text.size))] = 0xFF
        want_r, _ = orc.decode(text, mime=True)
        res = torch.empty(1, dtype=torch.int64, device="cuda")
        dst = torch.empty(b64.decoded_max_length(text.size), dtype=torch.uint8, device="cuda")
        b64.mime_decode_async(torch.from_numpy(text).cuda(), dst, res, std, ws)
        assert int(res.item()) == want_r, d
        if not hit[d]:
            assert want_r == 1 << 20


def test_bounded_wait_timeout_selftest(b64, orc):
    """The wait the kernels use for their bulk copies, on a barrier armed for a
    copy that is never issued: the call reports B64_E_TIMEOUT within the
    limit, the fault flag is raised, and the context keeps working."""
    import ctypes
    import time
    res = torch.zeros(1, dtype=torch.int64, device="cuda")
    t0 = time.time()
    rc = b64.lib().b64_selftest_wait_timeout(res.data_ptr(), ctypes.c_uint64(50_000_000),
                                             torch.cuda.current_stream().cuda_stream)
    assert rc == b64.B64_SUCCESS, b64.last_error()
    torch.cuda.synchronize()
    assert time.time() - t0 < 30
    assert int(res.item()) == b64.B64_E_TIMEOUT
    assert b64.device_fault_flag(clear=True) != 0
    assert b64.device_fault_flag() == 0
    rc = b64.lib().b64_selftest_wait_timeout(res.data_ptr(), ctypes.c_uint64(0), None)
    assert rc == b64.B64_ERR_INVALID_ARGUMENT
    text = wl.mime_wrap(orc.encode(wl.random_bytes(60_000, 800)))
    r, got = b64.mime_decode(torch.from_numpy(text).cuda(), b64.Alphabet.standard())
    assert r == 60_000


def test_stale_tile_memory_does_not_leak_into_seams(b64, orc):
    """A tile's last output byte comes from a group of four that the next tile
    finishes; the values past the tile's end are stale shared memory. Fill
    that memory with out-of-range values first (decode an all-bad input), then
    decode valid text whose tiles end mid-group: every byte must match."""
    std = b64.Alphabet.standard()
    junk = np.full(40 * TILE, ord("!"), np.uint8)
    r, _ = b64.mime_decode(torch.from_numpy(junk).cuda(), std)
    assert r == -1
    data = wl.random_bytes(24 << 20, 900)
    text = wl.mime_wrap(orc.encode(data))
    for _ in range(3):
        b64.mime_decode(torch.from_numpy(junk).cuda(), std)
        r, out = b64.mime_decode(torch.from_numpy(text).cuda(), std)
        assert r == data.size
        assert torch.equal(out, torch.from_numpy(data).cuda())


# ---- documents laid out as lines of L data characters + CR LF (L a multiple
#      of 4): the decode kernel's line fast path, and every way out of it

@pytest.mark.parametrize("L", [4, 12, 16, 20, 28, 64, 76, 1020])
@pytest.mark.parametrize("eol", [b"\r\n", b"\n"])
@pytest.mark.parametrize("src_off", [0, 3])
def test_line_layout_sizes(b64, orc, L, eol, src_off):
    std = b64.Alphabet.standard()
    for i, n in enumerate([3 * TILE, 3 * TILE + 1, 3 * TILE + 2, 200_000, 1_000_003]):
        text = wl.mime_wrap(orc.encode(wl.random_bytes(n, 700 + i)), line=L, eol=eol)
        if i % 2:
            text = np.concatenate([text, np.frombuffer(eol, np.uint8)])
        assert check(b64, orc, text, std, orc.standard_alphabet(), True, src_off=src_off,
                     strict_tail=True) == n


def test_line_layout_lf_broken(b64, orc):
    """LF-only lines: a data byte where an LF belongs, an LF replaced by a
    bad byte or by CR, an extra LF, a line one group short."""
    std, chars = b64.Alphabet.standard(), orc.standard_alphabet()
    good = wl.mime_wrap(orc.encode(wl.random_bytes(250_000, 730)), line=76, eol=b"\n")
    lfs = np.nonzero(good == 10)[0]
    g = wl.rng(731)
    for p in lfs[g.integers(0, lfs.size, 12)]:
        for v in (ord("Q"), 0x21, 13, 32):
            t = good.copy()
            t[int(p)] = v
            check(b64, orc, t, std, chars, True)
    p = int(lfs[40])
    check(b64, orc, np.concatenate([good[:p], np.frombuffer(b"\n", np.uint8), good[p:]]), std,
          chars, True)
    check(b64, orc, np.concatenate([good[:p - 4], good[p:]]), std, chars, True)


def test_line_layout_broken(b64, orc):
    """Errors and layout breaks in every position class of a 76-column
    document: a data byte, a CR or LF replaced (by data, by a bad byte, by
    a space), a line one group longer or shorter, '=' inside, a bad byte at
    a segment's first or last byte."""
    std, chars = b64.Alphabet.standard(), orc.standard_alphabet()
    data = wl.random_bytes(300_000, 710)
    good = wl.mime_wrap(orc.encode(data))
    m = good.size
    g = wl.rng(711)
    edits = []
    for seg in (0, 1, 7, 20, m // TILE - 1):
        base = seg * TILE
        for off in (0, 1, 2, 3, 75, 76, 77, 1000, TILE - 2, TILE - 1):
            p = base + off
            if p < m:
                edits += [(p, 0x21), (p, ord("A")), (p, ord(" ")), (p, ord("="))]
    for p in g.integers(0, m, 40):  # anywhere in a unit of four groups
        edits += [(int(p), 0x21), (int(p), ord("="))]
    crs = np.nonzero(good == 13)[0]
    for p in crs[g.integers(0, crs.size, 20)]:
        edits += [(int(p), ord("Q")), (int(p) + 1, ord("Q")), (int(p), 0xC3), (int(p), ord("\n"))]
    for p, v in edits:
        t = good.copy()
        t[p] = v
        check(b64, orc, t, std, chars, True)
    # one line a group longer, one a group shorter (every later segment shifts)
    lines = [good[k:k + 78] for k in range(0, m, 78)]
    for j, delta in ((3, 4), (100, -4), (600, 4)):
        t = [x.copy() for x in lines]
        if delta > 0:
            t[j] = np.concatenate([t[j][:76], np.frombuffer(b"ABCD", np.uint8), t[j][76:]])
        else:
            t[j] = np.concatenate([t[j][:72], t[j][76:]])
        check(b64, orc, np.concatenate(t), std, chars, True)


def test_line_layout_first_line_only(b64, orc):
    """The first line looks like the layout, the rest does not: spaces,
    LF-only breaks, random whitespace after the first line."""
    std, chars = b64.Alphabet.standard(), orc.standard_alphabet()
    text = orc.encode(wl.random_bytes(150_000, 720))
    head = wl.mime_wrap(text[:152])          # two 76-character lines
    rest = text[152:]
    for k, tail in enumerate([wl.insert_spaces(rest, seed=721, count=3000),
                              wl.mime_wrap(rest, line=76, eol=b"\n"),
                              wl.mime_wrap(rest, line=72)]):
        t = np.concatenate([head, np.frombuffer(b"\r\n", np.uint8), tail])
        assert check(b64, orc, t, std, chars, True) == 150_000, k


def test_line_layout_whole_extra_line(b64, orc):
    """An extra line of 76 spaces (and its CR LF) part way: every segment
    after it has its whitespace exactly where the 78-byte layout puts breaks,
    but 76 fewer data characters before it than the layout says. Only the
    segment holding the blank line breaks the layout; the result must still
    be the oracle's, with the counting path taking over. Also a blank line of
    another length, blank CR LF lines, and a whole line of data removed."""
    std, chars = b64.Alphabet.standard(), orc.standard_alphabet()
    data = wl.random_bytes(400_000, 740)
    good = wl.mime_wrap(orc.encode(data))
    for cut in (78 * 5, 78 * 300, 78 * 6000):
        for extra in (b" " * 76 + b"\r\n", b" " * 12 + b"\r\n", b"\r\n" * 39):
            t = np.concatenate([good[:cut], np.frombuffer(extra, np.uint8), good[cut:]])
            assert check(b64, orc, t, std, chars, True) == data.size
        t = np.concatenate([good[:cut], good[cut + 78:]])       # one whole line less
        assert check(b64, orc, t, std, chars, True) == data.size - 57


def test_call_recorded_in_a_cuda_graph(b64, orc):
    """The call's launch chain (status kernel, then five programmatic
    dependents) recorded once in a CUDA graph and replayed twice, on a
    document whose line layout holds (the one-pass kernel decodes it) and on
    one with a line a group longer part way (the counting kernels decode it
    again), each replay against the oracle."""
    std, chars = b64.Alphabet.standard(), orc.standard_alphabet()
    good = wl.mime_wrap(orc.encode(wl.random_bytes(700_000, 780)))
    lines = [good[k:k + 78] for k in range(0, good.size, 78)]
    lines[2000] = np.concatenate([lines[2000][:76], np.frombuffer(b"QUJD", np.uint8),
                                  lines[2000][76:]])
    broken = np.concatenate(lines)
    for text in (good, broken):
        want_r, want = orc.decode(text, chars, True, mime=True)
        src = torch.from_numpy(np.ascontiguousarray(text)).cuda()
        cap = b64.decoded_max_length(text.size)
        dst = torch.zeros(cap, dtype=torch.uint8, device="cuda")
        res = torch.zeros(1, dtype=torch.int64, device="cuda")
        ws = b64.mime_workspace(text.size)
        s = torch.cuda.Stream()
        b64.mime_decode_async(src, dst, res, std, ws, stream=s)   # first call sets up the kernels
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            b64.mime_decode_async(src, dst, res, std, ws, stream=s)
        for _ in range(2):
            dst.zero_()
            res.fill_(-7)
            torch.cuda.synchronize()
            g.replay()
            torch.cuda.synchronize()
            assert int(res.item()) == want_r
            if want_r >= 0:
                assert np.array_equal(dst[:want_r].cpu().numpy(), want)
