"""Parity of the batched (one persistent launch) codec with the oracle.

The workload is 100,000 independent strings with lognormal lengths (median
1 KiB, clipped to 1 B .. 1 MiB), half with the standard padded table and half
with base64url unpadded, every string checked byte for byte against the
oracle's batched loop; smaller cases cover every tile size, empty and tiny
strings, injected bad bytes, canaries between strings, CUDA-graph replay, and
identity with one launch per string.
"""
import numpy as np
import pytest
import torch

from paper_1910_05109_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def b64():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import __graft_entry__
    __graft_entry__.build()
    from paper_1910_05109_gb300 import binding
    binding.lib()
    yield binding
    assert binding.device_fault_flag() == 0


@pytest.fixture(scope="module")
def tables(b64, orc):
    return ([b64.Alphabet.standard(), b64.Alphabet.url()],
            orc.standard_alphabet() + orc.url_alphabet())


def make_batch(orc, count, seed, median=1024, sigma=1.5, hi=1 << 20, extra_lengths=()):
    lengths = wl.lognormal_lengths(count, seed, median, sigma, 1, hi)
    lengths = np.concatenate([lengths, np.asarray(extra_lengths, np.int64)])
    off = wl.offsets_from_lengths(lengths)
    data = wl.random_bytes(int(off[-1]), seed + 7)
    alph_id = wl.bernoulli(lengths.size, seed + 11).astype(np.uint8)  # 0 std padded, 1 url
    padded = (alph_id == 0).astype(np.int32)
    return data, off, alph_id, padded


def oracle_encode(orc, tables, data, off, alph_id, padded):
    elen = np.array([orc.encoded_length(int(off[i + 1] - off[i]), bool(padded[i]))
                     for i in range(off.size - 1)], np.int64)
    eoff = wl.offsets_from_lengths(elen)
    enc, res = orc.encode_batch(data, off, eoff, tables[1], alph_id.astype(np.int32), padded,
                                int(eoff[-1]))
    return enc, eoff, res


def gpu_encode(b64, tables, data, off, alph_id, units, src_shift=0, align16=False):
    dev = "cuda"
    buf = torch.empty(data.size + src_shift + 16, dtype=torch.uint8, device=dev)
    src = buf[src_shift:src_shift + data.size]
    if data.size:
        src.copy_(torch.from_numpy(data))
    d_off = torch.from_numpy(off).to(dev)
    d_aid = torch.from_numpy(alph_id).to(dev)
    dst_off = b64.batch_offsets(d_off, tables[0], d_aid, decode=False, align16=align16)
    total = int(dst_off[-1])
    dst = torch.full((total + 64,), 0xA5, dtype=torch.uint8, device=dev)
    res = b64.encode_batch(src, d_off, dst, dst_off, tables[0], d_aid, tile_units=units)
    torch.cuda.synchronize()
    host = dst.cpu().numpy()
    assert (host[total:] == 0xA5).all()
    return host[:total], dst_off.cpu().numpy(), res.cpu().numpy()


def gpu_decode(b64, tables, text, toff, alph_id, units, src_shift=0, align16=False):
    dev = "cuda"
    buf = torch.empty(text.size + src_shift + 16, dtype=torch.uint8, device=dev)
    src = buf[src_shift:src_shift + text.size]
    if text.size:
        src.copy_(torch.from_numpy(text))
    d_off = torch.from_numpy(toff).to(dev)
    d_aid = torch.from_numpy(alph_id).to(dev)
    dst_off = b64.batch_offsets(d_off, tables[0], d_aid, decode=True, align16=align16)
    total = int(dst_off[-1])
    dst = torch.full((total + 64,), 0xA5, dtype=torch.uint8, device=dev)
    res = b64.decode_batch(src, d_off, dst, dst_off, tables[0], d_aid, tile_units=units)
    torch.cuda.synchronize()
    return dst.cpu().numpy(), dst_off.cpu().numpy(), res.cpu().numpy()


def check_decoded(host, dst_off, res, want_res, want_dec):
    """Results equal the oracle's; each decoded string equals the oracle's bytes
    at the same offsets, with nothing written past it up to its capacity."""
    assert np.array_equal(res, want_res)
    for i in range(res.size):
        o = int(dst_off[i])
        if res[i] >= 0:
            assert np.array_equal(host[o:o + res[i]], want_dec[o:o + res[i]]), i
            assert (host[o + res[i]:int(dst_off[i + 1])] == 0xA5).all(), i


EDGE_LENGTHS = [0, 1, 2, 3, 4, 5, 0, 0, 383, 384, 385, 767, 768, 769, 1535, 1536, 1537,
                3071, 3072, 3073, 4096, 100_000, 0]


PAIRS = 1 << 16   # B64_TILE_PAIRS: encode's whole 8-unit tiles through pair tables


@pytest.mark.parametrize("units", [1, 2, 4, 8, 8 | PAIRS])
def test_batch_parity_all_tiles(b64, orc, tables, units):
    data, off, aid, padded = make_batch(orc, 1500, seed=20 + units, hi=1 << 17,
                                        extra_lengths=EDGE_LENGTHS)
    want, eoff, wres = oracle_encode(orc, tables, data, off, aid, padded)
    got, goff, gres = gpu_encode(b64, tables, data, off, aid, units, src_shift=units % 3)
    assert np.array_equal(goff, eoff)
    assert np.array_equal(gres, wres)
    assert np.array_equal(got, want)
    dec, doff, dres = gpu_decode(b64, tables, want, eoff, aid, units, src_shift=(units + 1) % 5)
    want_dec, want_res = orc.decode_batch(want, eoff, doff, tables[1], aid.astype(np.int32),
                                          padded, int(doff[-1]))
    assert np.array_equal(want_res, off[1:] - off[:-1])
    check_decoded(dec, doff, dres, want_res, want_dec)


@pytest.mark.parametrize("units", [1, 4, 8 | PAIRS])
def test_batch_parity_aligned_offsets(b64, orc, tables, units):
    """Output offsets with 16-byte aligned string starts (the kernels store
    such outputs straight from registers): every string equals the oracle's,
    the bytes between strings are untouched, and decode results and bytes
    (aligned offsets too, with injected bad bytes) equal the oracle's."""
    data, off, aid, padded = make_batch(orc, 1500, seed=40 + units, hi=1 << 17,
                                        extra_lengths=EDGE_LENGTHS)
    want, eoff, wres = oracle_encode(orc, tables, data, off, aid, padded)
    got, goff, gres = gpu_encode(b64, tables, data, off, aid, units, src_shift=units % 3,
                                 align16=True)
    assert np.array_equal(gres, wres)
    assert (goff % 16 == 0).all()
    for i in range(off.size - 1):
        a, m = int(goff[i]), int(wres[i])
        assert np.array_equal(got[a:a + m], want[eoff[i]:eoff[i] + m]), i
        assert (got[a + m:int(goff[i + 1])] == 0xA5).all(), i
    text = want.copy()
    g = wl.rng(44 + units)
    for i in np.nonzero(g.random(off.size - 1) < 0.05)[0]:
        if eoff[i + 1] > eoff[i]:
            text[eoff[i] + int(g.integers(0, eoff[i + 1] - eoff[i]))] = 0xFF
    dec, doff, dres = gpu_decode(b64, tables, text, eoff, aid, units, align16=True)
    assert (doff % 16 == 0).all()
    want_dec, want_res = orc.decode_batch(text, eoff, doff, tables[1], aid.astype(np.int32),
                                          padded, int(doff[-1]))
    assert (want_res < 0).sum() > 10
    check_decoded(dec, doff, dres, want_res, want_dec)


def test_batch_injected_errors(b64, orc, tables):
    data, off, aid, padded = make_batch(orc, 2000, seed=31, hi=1 << 16,
                                        extra_lengths=EDGE_LENGTHS)
    text, eoff, _ = oracle_encode(orc, tables, data, off, aid, padded)
    text = text.copy()
    g = wl.rng(32)
    hit = g.random(off.size - 1) < 0.05
    for i in np.nonzero(hit)[0]:
        m = int(eoff[i + 1] - eoff[i])
        if m:
            # a bad byte, or a misplaced '=', anywhere in the string
            v = int(g.choice([0x00, 0x0A, 0x2D, 0x2B, 0x3D, 0x7F, 0xC3, 0xFF]))
            text[eoff[i] + int(g.integers(0, m))] = v
    for units in (1, 4):
        dec, doff, dres = gpu_decode(b64, tables, text, eoff, aid, units)
        want_dec, want_res = orc.decode_batch(text, eoff, doff, tables[1], aid.astype(np.int32),
                                              padded, int(doff[-1]))
        assert (want_res < 0).sum() > 50
        check_decoded(dec, doff, dres, want_res, want_dec)


def test_batch_single_and_empty(b64, orc, tables):
    for lengths in ([0], [1], [2], [3], [5000], [0, 0, 7, 0]):
        off = wl.offsets_from_lengths(np.array(lengths, np.int64))
        data = wl.random_bytes(int(off[-1]), 40)
        aid = np.zeros(len(lengths), np.uint8)
        padded = np.ones(len(lengths), np.int32)
        want, eoff, wres = oracle_encode(orc, tables, data, off, aid, padded)
        got, goff, gres = gpu_encode(b64, tables, data, off, aid, 4)
        assert np.array_equal(got, want) and np.array_equal(gres, wres)
        dec, doff, dres = gpu_decode(b64, tables, want, eoff, aid, 4)
        want_dec, want_res = orc.decode_batch(want, eoff, doff, tables[1], aid.astype(np.int32),
                                              padded, int(doff[-1]))
        check_decoded(dec, doff, dres, want_res, want_dec)
    # n == 0 enqueues nothing
    z = torch.zeros(1, dtype=torch.int64, device="cuda")
    b64.encode_batch(torch.zeros(1, dtype=torch.uint8, device="cuda"), z,
                     torch.zeros(1, dtype=torch.uint8, device="cuda"), z, tables[0])


def test_batch_tiny_strings_and_offset_origin(b64, orc, tables):
    """20,000 strings of 0..9 bytes (far fewer bytes than the grid has warps,
    so most warps' byte ranges are empty or end inside a string's first
    group), with src_off starting past 0 (bytes before the first string are
    not part of the batch); then the same for decode, where strings of 0..13
    characters are mostly tail (handled by the finalize kernel)."""
    g = wl.rng(50)
    lengths = g.integers(0, 10, 20_000).astype(np.int64)
    origin = 37
    off = wl.offsets_from_lengths(lengths) + origin
    data = wl.random_bytes(int(off[-1]), 51)
    aid = wl.bernoulli(lengths.size, 52).astype(np.uint8)
    padded = (aid == 0).astype(np.int32)
    want, eoff, wres = oracle_encode(orc, tables, data, off, aid, padded)
    for units in (1, 8):
        got, goff, gres = gpu_encode(b64, tables, data, off, aid, units)
        assert np.array_equal(gres, wres)
        assert np.array_equal(goff - goff[0], eoff - eoff[0])
        assert np.array_equal(got, want)
    text = np.concatenate([wl.random_bytes(origin, 53), want])
    toff = eoff + origin
    for units in (2, 4):
        dec, doff, dres = gpu_decode(b64, tables, text, toff, aid, units)
        want_dec, want_res = orc.decode_batch(text, toff, doff, tables[1], aid.astype(np.int32),
                                              padded, int(doff[-1]))
        assert np.array_equal(want_res, lengths)
        check_decoded(dec, doff, dres, want_res, want_dec)


@pytest.mark.parametrize("align16", [False, True])
def test_batch_config3_full_size(b64, orc, tables, align16):
    """100,000 strings, lognormal lengths (median 1 KiB, sigma 1.5, 1 B..1 MiB),
    all three residues mod 3, 50/50 standard-padded / url-unpadded, 1% of the
    decode inputs with one injected bad byte: every string against the oracle,
    with packed output offsets and with 16-byte aligned string starts (the
    benchmark's layout)."""
    data, off, aid, padded = make_batch(orc, 100_000, seed=2)
    lens = off[1:] - off[:-1]
    assert set(np.unique(lens % 3)) == {0, 1, 2}
    want, eoff, wres = oracle_encode(orc, tables, data, off, aid, padded)
    got, goff, gres = gpu_encode(b64, tables, data, off, aid, 4, align16=align16)
    assert np.array_equal(gres, wres)
    if align16:
        keep = np.zeros(got.size, bool)
        for i in range(off.size - 1):
            keep[goff[i]:goff[i] + wres[i]] = True
        assert np.array_equal(got[keep], want)
        assert (got[~keep] == 0xA5).all()
    else:
        assert np.array_equal(got, want)
    text = want.copy()
    g = wl.rng(12)
    bad = np.nonzero(g.random(off.size - 1) < 0.01)[0]
    for i in bad:
        m = int(eoff[i + 1] - eoff[i])
        p = int(g.integers(0, m))
        text[eoff[i] + p] = 0xFF
    dec, doff, dres = gpu_decode(b64, tables, text, eoff, aid, 4, align16=align16)
    want_dec, want_res = orc.decode_batch(text, eoff, doff, tables[1], aid.astype(np.int32),
                                          padded, int(doff[-1]))
    assert (want_res < 0).sum() == bad.size
    assert np.array_equal(dres, want_res)
    ok = want_res >= 0
    for i in np.nonzero(ok)[0][::97]:
        o = int(doff[i])
        assert np.array_equal(dec[o:o + want_res[i]], data[off[i]:off[i + 1]])
    # all valid strings' bytes, compared at once through the oracle's output
    mask = np.zeros(dec.size, bool)
    for i in np.nonzero(ok)[0]:
        mask[doff[i]:doff[i] + want_res[i]] = True
    assert np.array_equal(dec[:want_dec.size][mask[:want_dec.size]],
                          want_dec[mask[:want_dec.size]])


def test_batch_graph_and_per_string_identity(b64, orc, tables):
    data, off, aid, padded = make_batch(orc, 400, seed=50, hi=1 << 15)
    d_src = torch.from_numpy(data).cuda()
    d_off = torch.from_numpy(off).cuda()
    d_aid = torch.from_numpy(aid).cuda()
    dst_off = b64.batch_offsets(d_off, tables[0], d_aid, decode=False)
    total = int(dst_off[-1])
    dst = torch.zeros(total, dtype=torch.uint8, device="cuda")
    ws = b64.batch_workspace(off.size - 1)
    res = torch.empty(off.size - 1, dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    b64.encode_batch(d_src, d_off, dst, dst_off, tables[0], d_aid, res, 2, ws, stream=s)
    torch.cuda.synchronize()
    first = dst.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b64.encode_batch(d_src, d_off, dst, dst_off, tables[0], d_aid, res, 2, ws, stream=s)
    dst.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(dst, first)
    # one launch per string through the single-buffer call: identical bytes
    per = torch.zeros_like(dst)
    hoff = dst_off.cpu().numpy()
    alph = tables[0]
    for i in range(off.size - 1):
        if off[i + 1] > off[i]:
            b64.encode(d_src[off[i]:off[i + 1]], alph[aid[i]], per[hoff[i]:hoff[i + 1]])
    torch.cuda.synchronize()
    assert torch.equal(per, first)


def test_batch_codec_graph_and_autotune_cache(b64, orc, tables, tmp_path):
    from paper_1910_05109_gb300 import autotune
    from paper_1910_05109_gb300.batch import BatchCodec
    data, off, aid, padded = make_batch(orc, 800, seed=70, hi=1 << 14)
    want, eoff, _ = oracle_encode(orc, tables, data, off, aid, padded)
    n = off.size - 1
    codec = BatchCodec("encode", n, data.size, tables[0])
    total = codec.load(torch.from_numpy(data).cuda(), torch.from_numpy(off).cuda(),
                       torch.from_numpy(aid).cuda())
    assert total == want.size
    path = str(tmp_path / "autotune.json")
    args = (codec.src, codec.src_off, codec.dst, codec.dst_off, tables[0], codec.alph_id[:n])
    units, timings = autotune.best_units("encode", *args, path=path)
    choices = autotune.choices("encode", len(tables[0]))   # two alphabets: pair tables too
    assert units in choices and set(timings) == set(choices) and len(choices) == 12
    again, t2 = autotune.best_units("encode", *args, path=path)
    assert again == units and t2 == {}          # served from the cache file
    codec.tile_units = units
    for _ in range(3):                          # first call direct, then graph replays
        with torch.cuda.stream(codec.stream):
            codec.dst.zero_()
        codec.run()
        codec.synchronize()
        assert np.array_equal(codec.dst[:total].cpu().numpy(), want)
