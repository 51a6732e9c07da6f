"""Parity of the CUDA codec with the oracle, through the C ABI.

Bit-exact comparisons on seeded inputs: sizes that span several chunks and
ragged tails, every alignment class, both alphabets and a custom one, canary
bytes after the output, error offsets for injected bad bytes, the strict
rules, brute force over all 2^24 triples, and the full-size 1 GiB buffers on
sampled windows plus properties that hold at any size.
"""
import numpy as np
import pytest
import torch

from conftest import read_golden
from paper_1910_05109_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

ENC_CHUNK = 384     # input bytes per warp chunk of the encode kernel below 32 MiB
ENC_LARGE_MIN = 32 << 20   # from here on: 1152-byte warp chunks, bulk stores
ENC_LARGE_CHUNK = 1152
DEC_CHUNK = 2048    # characters per warp chunk of the decode body kernel below 64 MiB
DEC_WARPS = 16      # warps per block of the decode body kernel (one block per SM)
# (characters per warp chunk, input buffers per warp) below and from 64 MiB
DEC_SHAPES = {"small": (2048, 4), "large": (1024, 8)}
DEC_LARGE_MIN = 64 << 20


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
def alphabets(b64, orc):
    std, url = b64.Alphabet.standard(), b64.Alphabet.url()
    rev = orc.standard_alphabet()[::-1]
    custom = b64.Alphabet.create(rev, True)
    custom_np = b64.Alphabet.create(rev, False)
    return {
        "std": (std, orc.standard_alphabet(), True),
        "url": (url, orc.url_alphabet(), False),
        "url_padded": (b64.Alphabet.create(orc.url_alphabet(), True), orc.url_alphabet(), True),
        "custom": (custom, rev, True),
        "custom_unpadded": (custom_np, rev, False),
    }


def to_dev(arr: np.ndarray, offset: int = 0, slack: int = 64) -> torch.Tensor:
    """Device copy of arr starting `offset` bytes past a 256-byte boundary."""
    buf = torch.empty(arr.size + offset + slack, dtype=torch.uint8, device="cuda")
    view = buf[offset:offset + arr.size]
    if arr.size:
        view.copy_(torch.from_numpy(np.ascontiguousarray(arr)))
    return view


def canvas(cap: int, offset: int = 0, slack: int = 64):
    """Output buffer filled with 0xA5; returns (whole buffer, view at offset)."""
    buf = torch.full((cap + offset + slack,), 0xA5, dtype=torch.uint8, device="cuda")
    return buf, buf[offset:offset + max(cap, 1)]


def check_canary(buf: torch.Tensor, offset: int, written: int):
    host = buf.cpu().numpy()
    assert (host[:offset] == 0xA5).all(), "bytes before dst were written"
    assert (host[offset + written:] == 0xA5).all(), "bytes past the output length were written"


def gpu_encode(b64, data, alph, src_off=0, dst_off=0):
    src = to_dev(data, src_off)
    cap = b64.encoded_length(data.size, alph.padded)
    buf, dst = canvas(cap, dst_off)
    out = b64.encode(src, alph, dst)
    torch.cuda.synchronize()
    check_canary(buf, dst_off, out.numel())
    return out.cpu().numpy()


def gpu_decode(b64, text, alph, src_off=0, dst_off=0):
    src = to_dev(text, src_off)
    cap = b64.decoded_max_length(text.size)
    buf, dst = canvas(cap, dst_off)
    r, out = b64.decode(src, alph, dst)
    check_canary(buf, dst_off, r if r >= 0 else cap)
    return r, out.cpu().numpy()


SIZES = sorted(set(
    list(range(0, 70)) + [95, 96, 97, 255, 256, 257, 1000, 4095, 4096, 4097] +
    [k * ENC_CHUNK + d for k in (1, 2, 3, 7) for d in (-3, -2, -1, 0, 1, 2, 3)] +
    [k * DEC_CHUNK // 4 * 3 + d for k in (1, 2, 5) for d in (-4, -1, 0, 1, 4)] +
    list(wl.TABLE2_SIZES[:3]) + [1_048_575, 1_048_576, 1_048_577, 3_000_001] +
    # encoded length around 32 KiB (one block / a cluster of blocks), 64 KiB
    # and 128 KiB (8 and 16 blocks of 8 KiB) and 512 KiB (one cluster / the
    # three-launch decode)
    [24_573, 24_574, 24_575, 24_576, 24_577, 24_579,
     49_149, 49_150, 49_151, 49_152, 49_153, 49_155, 98_304, 98_305, 98_307,
     393_213, 393_215, 393_216, 393_217, 393_219]))


@pytest.mark.parametrize("name", ["std", "url", "url_padded", "custom", "custom_unpadded"])
def test_encode_decode_parity_sizes(b64, orc, alphabets, name):
    alph, chars, padded = alphabets[name]
    for i, n in enumerate(SIZES):
        data = wl.random_bytes(n, seed=1000 + i)
        want = orc.encode(data, chars, padded)
        got = gpu_encode(b64, data, alph)
        assert np.array_equal(got, want), (name, n)
        r_want, d_want = orc.decode(want, chars, padded)
        r, d = gpu_decode(b64, want, alph)
        assert r == r_want == n, (name, n, r)
        assert np.array_equal(d, d_want), (name, n)


@pytest.mark.parametrize("name", ["std", "url"])
def test_encode_large_shape(b64, orc, alphabets, name):
    """Sizes around the switch to the large encode shape, and one where every
    warp refills its seven input buffers twice with a ragged remainder;
    bit-exact against the oracle, then decoded back."""
    alph, chars, padded = alphabets[name]
    gw = torch.cuda.get_device_properties(0).multi_processor_count * 16
    for i, n in enumerate((ENC_LARGE_MIN - 1, ENC_LARGE_MIN, ENC_LARGE_MIN + 2,
                           ENC_LARGE_CHUNK * gw * 14 + ENC_LARGE_CHUNK - 1)):
        data = wl.random_bytes(n, seed=5000 + i)
        want = orc.encode(data, chars, padded)
        got = gpu_encode(b64, data, alph)
        assert np.array_equal(got, want), (name, n)
        r, d = gpu_decode(b64, want, alph)
        assert r == n and np.array_equal(d, data), (name, n)


def test_config1_single_buffer(b64, orc, alphabets):
    # 2^20 - 1 bytes of seed 0 (and the two sizes that give '=' and '==').
    alph, chars, padded = alphabets["std"]
    for n in (1_048_575, 1_048_576, 1_048_577):
        data = wl.random_bytes(n, seed=0)
        want = orc.encode(data, chars, padded)
        got = gpu_encode(b64, data, alph)
        assert np.array_equal(got, want)
        r, d = gpu_decode(b64, want, alph)
        assert r == n and np.array_equal(d, orc.decode(want, chars, padded)[1])


@pytest.mark.parametrize("src_off", [0, 1, 2, 3, 4, 8, 15])
@pytest.mark.parametrize("dst_off", [0, 1, 4, 13])
def test_alignment_classes(b64, orc, alphabets, src_off, dst_off):
    alph, chars, padded = alphabets["std"]
    # up to 512 KiB of characters decode in one launch; 600,001 bytes take the
    # three-launch path (the generic kernel when src or dst is unaligned)
    for i, n in enumerate((0, 1, 2, 5, 1000, 3 * ENC_CHUNK + 2, 50_001, 600_001)):
        data = wl.random_bytes(n, seed=2000 + i)
        want = orc.encode(data, chars, padded)
        assert np.array_equal(gpu_encode(b64, data, alph, src_off, dst_off), want), n
        r, d = gpu_decode(b64, want, alph, src_off, dst_off)
        assert r == n and np.array_equal(d, data), n
        bad, off, _ = wl.inject_invalid(want, seed=3000 + i, alphabet=chars)
        if bad.size:
            assert gpu_decode(b64, bad, alph, src_off, dst_off)[0] == orc.decode(bad, chars,
                                                                                  padded)[0]


def test_injected_invalid_byte_offsets(b64, orc, alphabets):
    alph, chars, padded = alphabets["std"]
    data = wl.random_bytes(7 * ENC_CHUNK + 1, seed=11)
    text = orc.encode(data, chars, padded)
    for seed in range(60):
        bad, off, val = wl.inject_invalid(text, seed=seed, alphabet=chars)
        want = orc.decode(bad, chars, padded)[0]
        assert gpu_decode(b64, bad, alph)[0] == want, (off, val)
        if off < bad.size - 2:
            assert want == -(off + 1)


@pytest.mark.parametrize("chunks", [64, 4000])  # one-launch decode / body kernel + tail kernel
def test_invalid_bytes_at_chunk_edges(b64, orc, alphabets, chunks):
    alph, chars, padded = alphabets["std"]
    text = orc.encode(wl.random_bytes(chunks // 4 * 3 * DEC_CHUNK, seed=12), chars, padded)
    m = text.size
    positions = [0, 1, 15, 16, DEC_CHUNK - 1, DEC_CHUNK, DEC_CHUNK + 1, 2 * DEC_CHUNK - 5,
                 3 * DEC_CHUNK + 7, m - DEC_CHUNK - 1, m - DEC_CHUNK, m - 7, m - 6, m - 5,
                 m - 4, m - 3, m - 2, m - 1]
    values = [0x00, 0x0A, 0x20, 0x2D, 0x3D, 0x5F, 0x7F, 0x80, 0xC3, 0xFF]
    for p in positions:
        for v in values:
            bad = text.copy()
            bad[p] = v
            assert gpu_decode(b64, bad, alph)[0] == orc.decode(bad, chars, padded)[0], (p, v)
    # Two bad bytes in different chunks: the smaller offset wins.
    bad = text.copy()
    bad[3 * DEC_CHUNK + 5] = 0xFF
    bad[DEC_CHUNK + 9] = ord("-")
    assert gpu_decode(b64, bad, alph)[0] == -(DEC_CHUNK + 10)


@pytest.mark.parametrize("shape", ["small", "large"])
def test_errors_in_refilled_stages(b64, orc, alphabets, shape):
    """Enough chunks that every warp refills each of its input buffers several
    times; bad bytes anywhere in a chunk (not only in lane 0's unit) must be
    found while the refill of the same buffer is pending, in the first and
    last chunk of a warp's first pass and in later passes. Both body shapes."""
    alph, chars, padded = alphabets["std"]
    chunk, stages = DEC_SHAPES[shape]
    gw = torch.cuda.get_device_properties(0).multi_processor_count * DEC_WARPS
    n_chunks = stages * gw * 3 + 5
    if shape == "large":
        n_chunks = max(n_chunks, DEC_LARGE_MIN // chunk + 5)
    else:
        assert n_chunks * chunk < DEC_LARGE_MIN
    text = orc.encode(wl.random_bytes(3 * chunk // 4 * n_chunks, seed=15), chars, padded)
    dev = to_dev(text)
    for c in (0, 1, 2, gw - 1, gw, gw + 1, stages * gw - 1, stages * gw, stages * gw + 1,
              2 * stages * gw + 77, n_chunks - 2):
        for inner in (0, 17, 511, 512, chunk - 24, chunk - 1):
            pos = c * chunk + inner
            t = dev.clone()
            t[pos] = 0x18
            r, _ = b64.decode(t, alph)
            assert r == -(pos + 1), (c, inner, r)
    r, out = b64.decode(dev, alph)
    assert r == 3 * chunk // 4 * n_chunks
    assert np.array_equal(out.cpu().numpy(), orc.decode(text, chars, padded)[1])


def test_every_byte_value_rejected(b64, orc, alphabets):
    alph, chars, padded = alphabets["std"]
    text = orc.encode(wl.random_bytes(3000, seed=13), chars, padded)
    members = set(chars)
    for v in range(256):
        for p in (0, 17, 2001, text.size - 3):
            bad = text.copy()
            bad[p] = v
            r = gpu_decode(b64, bad, alph)[0]
            want = orc.decode(bad, chars, padded)[0]
            assert r == want, (v, p)
            if v not in members:
                assert r == -(p + 1)


def test_strict_readings_on_gpu(b64, orc, alphabets):
    for mode, hexin, result, _ in read_golden("strict_readings.txt"):
        if mode == "mime":
            continue
        name = "std" if mode == "padded" else "url"
        alph, chars, padded = alphabets[name]
        src = np.frombuffer(b"" if hexin == "-" else bytes.fromhex(hexin), np.uint8)
        if name == "url":
            # the fixture's unpadded cases use characters common to both tables
            assert not set(src.tolist()) & {ord("+"), ord("/")}
        r, out = gpu_decode(b64, src, alph)
        want_r, want = orc.decode(src, chars, padded)
        assert r == want_r == int(result), (mode, hexin)
        if r >= 0:
            assert np.array_equal(out, want)


@pytest.mark.parametrize("name", ["std", "url"])
def test_random_mutations(b64, orc, alphabets, name):
    alph, chars, padded = alphabets[name]
    g = wl.rng(14)
    for i in range(400):
        n = int(g.integers(0, 200))
        text = orc.encode(wl.random_bytes(n, seed=4000 + i), chars, padded).copy()
        k = int(g.integers(0, 3))
        for _ in range(k):
            if text.size:
                text[int(g.integers(0, text.size))] = int(g.integers(0, 256))
        if g.random() < 0.3 and text.size:
            text = np.delete(text, int(g.integers(0, text.size)))
        want_r, want = orc.decode(text, chars, padded)
        r, out = gpu_decode(b64, text, alph)
        assert r == want_r, (i, text.tobytes())
        if r >= 0:
            assert np.array_equal(out, want)


def test_all_triples_bruteforce(b64, orc, alphabets):
    alph, chars, padded = alphabets["std"]
    v = np.arange(1 << 24, dtype=np.uint32)
    data = np.stack([(v >> 16) & 255, (v >> 8) & 255, v & 255], axis=1).astype(np.uint8).ravel()
    want = orc.encode(data, chars, padded)
    src = to_dev(data)
    out = b64.encode(src, alph)
    assert torch.equal(out, torch.from_numpy(want).cuda())
    r, dec = b64.decode(torch.from_numpy(want).cuda(), alph)
    assert r == data.size and torch.equal(dec, src)


def test_all_short_tails(b64, orc, alphabets):
    # Every 1- and 2-byte input after a 3-byte prefix (tail path, both modes).
    for name in ("std", "url"):
        alph, chars, padded = alphabets[name]
        for t in range(256 + 65536):
            if name == "url" and t >= 256 and t % 7:
                continue
            tail = [t] if t < 256 else [(t - 256) >> 8, (t - 256) & 255]
            data = np.array([7, 8, 9] + tail, np.uint8)
            want = orc.encode(data, chars, padded)
            assert np.array_equal(gpu_encode(b64, data, alph), want), (name, tail)
            if t % 97 == 0:
                r, d = gpu_decode(b64, want, alph)
                assert r == data.size and np.array_equal(d, data)


def test_decode_async_graph_and_streams(b64, orc, alphabets):
    alph, chars, padded = alphabets["url"]
    data = [wl.random_bytes(n, seed=5000 + n) for n in (123_457, 1_000_003)]
    texts = [orc.encode(d, chars, padded) for d in data]
    srcs = [to_dev(t) for t in texts]
    dsts = [torch.empty(b64.decoded_max_length(t.size), dtype=torch.uint8, device="cuda")
            for t in texts]
    res = torch.empty(2, dtype=torch.int64, device="cuda")
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    for i in range(2):
        b64.decode_async(srcs[i], dsts[i], res[i:i + 1], alph, streams[i])
    torch.cuda.synchronize()
    for i in range(2):
        assert int(res[i]) == data[i].size
        assert np.array_equal(dsts[i][:data[i].size].cpu().numpy(), data[i])
    # Encode + decode recorded in a CUDA graph and replayed.
    enc_out = torch.empty(b64.encoded_length(data[1].size, padded), dtype=torch.uint8,
                          device="cuda")
    src = to_dev(data[1])
    s = torch.cuda.Stream()
    b64.encode(src, alph, enc_out, stream=s)     # first call sets up the kernels
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        b64.encode(src, alph, enc_out, stream=s)
        b64.decode_async(enc_out, dsts[1], res[1:2], alph, stream=s)
    enc_out.zero_()
    dsts[1].zero_()
    res.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(enc_out.cpu().numpy(), texts[1])
    assert int(res[1]) == data[1].size
    assert np.array_equal(dsts[1][:data[1].size].cpu().numpy(), data[1])


def test_full_size_64mib_and_1gib(b64, orc, alphabets):
    """The large single-buffer workload (64 MiB and 1 GiB of seed-1 random
    bytes, standard and url tables swapped at run time): full oracle parity at
    64 MiB; at 1 GiB the oracle encodes the whole buffer once, and the GPU
    output is compared byte for byte, decoded back and checked for the
    injected-error offset."""
    for n, seed in ((64 << 20, 1), (1 << 30, 1)):
        data = wl.random_bytes(n, seed=seed)
        src = torch.from_numpy(data).cuda()
        for name in ("std", "url_padded"):
            alph, chars, padded = alphabets[name]
            want = orc.encode(data, chars, padded)
            want_dev = torch.from_numpy(want).cuda()
            out = b64.encode(src, alph)
            assert out.numel() == want.size
            assert torch.equal(out, want_dev), (n, name)
            del out
            r, dec = b64.decode(want_dev, alph)
            assert r == n and torch.equal(dec, src), (n, name)
            # Sampled decode windows against the oracle's own decode.
            g = wl.rng(seed + 17)
            for _ in range(8):
                q = int(g.integers(0, want.size // 4 - 1000))
                w = want[4 * q:4 * q + 4000]
                assert np.array_equal(dec[3 * q:3 * q + 3000].cpu().numpy(), orc.decode(w, chars)[1])
            del dec
            bad, off, val = wl.inject_invalid(want, seed=11, alphabet=chars)
            want_r = orc.decode(bad, chars, padded)[0] if n < (1 << 30) else -(off + 1)
            if n >= (1 << 30):
                assert off < bad.size - 2   # outside the padding zone: the offset is exact
            r, _ = b64.decode(torch.from_numpy(bad).cuda(), alph)
            assert r == want_r, (n, name, off, val)
            del want_dev, bad
        del src
        torch.cuda.empty_cache()
