"""Canonical mode (B64_FLAG_CANONICAL, reading R7) on every decode path,
against the oracle: the single-buffer decode at sizes that take the one-block,
the cluster and the three-launch paths, the batched decode (every "XYZ=" and
mixed alphabets), the MIME decode and the host-buffer codec. Inputs are valid
encodings whose last data character gets non-zero unused bits."""
import numpy as np
import pytest
import torch

from paper_1910_05109_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

STD = b"ABCDEFGHIJKLMNOPQRSTUVWXYZabcdefghijklmnopqrstuvwxyz0123456789+/"
URL = STD[:62] + b"-_"


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
def alphs(b64):
    std_c = b64.Alphabet.create(STD, True, canonical=True)
    url_c = b64.Alphabet.create(URL, False, canonical=True)
    assert std_c.canonical and std_c.padded and url_c.canonical and not url_c.padded
    assert not b64.Alphabet.standard().canonical
    return {"std": (std_c, STD, True), "url": (url_c, URL, False)}


def spoil(text: np.ndarray, chars: bytes, bit: int):
    """Sets unused low bits (bit & mask) of the last data character if the
    final group is partial; returns (copy, whether a bit was set)."""
    t = text.copy()
    k = t.size
    while k and t[k - 1] == ord("="):
        k -= 1
    if k % 4 in (2, 3):
        v = chars.index(bytes([t[k - 1]]))
        low = 15 if k % 4 == 2 else 3
        t[k - 1] = chars[v | (bit & low)]
        return t, (bit & low) != 0
    return t, False


def spoil_last(text: np.ndarray, chars: bytes, padded: bool, bit: int) -> np.ndarray:
    return spoil(text, chars, bit)[0]


SIZES = [1, 2, 4, 5, 1000, 1001, 49_150, 49_151, 200_000, 200_001, 393_215, 393_217,
         1_000_000, 1_000_001]


@pytest.mark.parametrize("name", ["std", "url"])
def test_single_buffer(b64, orc, alphs, name):
    alph, chars, padded = alphs[name]
    for i, n in enumerate(SIZES):
        data = wl.random_bytes(n, 70 + i)
        text = orc.encode(data, chars, padded)
        for bit in (0, 1, 2, 8):
            t, spoiled = spoil(text, chars, bit)
            want_r, want = orc.decode(t, chars, padded, canonical=True)
            r, out = b64.decode(torch.from_numpy(t).cuda(), alph)
            assert r == want_r, (name, n, bit, r, want_r)
            assert (r < 0) == spoiled
            if r >= 0:
                assert np.array_equal(out.cpu().numpy(), want)


def test_batch_every_final_group_and_mixed(b64, orc, alphs):
    # every "XYZ=" string with the canonical standard table
    v = np.arange(256 ** 3, dtype=np.uint32)
    strings = np.stack([(v >> 16) & 255, (v >> 8) & 255, v & 255,
                        np.full(v.size, ord("="))], axis=1).astype(np.uint8)
    n = strings.shape[0]
    off = np.arange(n + 1, dtype=np.int64) * 4
    doff = np.arange(n + 1, dtype=np.int64) * 3
    _, want = orc.decode_batch(strings.ravel(), off, doff, STD, np.zeros(n, np.int32),
                               np.full(n, 3, np.int32), 3 * n)
    dst = torch.zeros(3 * n + 16, dtype=torch.uint8, device="cuda")
    got = b64.decode_batch(torch.from_numpy(strings.ravel()).cuda(), torch.from_numpy(off).cuda(),
                           dst, torch.from_numpy(doff).cuda(), [alphs["std"][0]]).cpu().numpy()
    assert np.array_equal(got, want)
    assert (want == 2).sum() == 64 * 64 * 16 and (want == 1).sum() == 64 * 4

    # mixed: canonical standard and plain base64url, spoiled and clean strings
    g = wl.rng(71)
    lens = g.integers(0, 300, 3000)
    aid = (g.random(lens.size) < 0.5).astype(np.uint8)
    texts = []
    for i, L in enumerate(lens):
        chars, padded = (STD, True) if aid[i] == 0 else (URL, False)
        t = orc.encode(wl.random_bytes(int(L), 1000 + i), chars, padded)
        texts.append(spoil_last(t, chars, padded, int(g.integers(0, 4))))
    toff = np.concatenate([[0], np.cumsum([t.size for t in texts])]).astype(np.int64)
    text = np.concatenate(texts) if texts else np.zeros(0, np.uint8)
    doff = np.concatenate([[0], np.cumsum([(t.size + 3) // 4 * 3 for t in texts])]).astype(np.int64)
    flags = np.where(aid == 0, 3, 0).astype(np.int32)  # url here: not canonical
    want_dec, want_res = orc.decode_batch(text, toff, doff, STD + URL, aid.astype(np.int32), flags,
                                          int(doff[-1]))
    dst = torch.zeros(int(doff[-1]) + 16, dtype=torch.uint8, device="cuda")
    res = b64.decode_batch(torch.from_numpy(text).cuda(), torch.from_numpy(toff).cuda(), dst,
                           torch.from_numpy(doff).cuda(), [alphs["std"][0], b64.Alphabet.url()],
                           torch.from_numpy(aid).cuda()).cpu().numpy()
    assert np.array_equal(res, want_res)
    assert (want_res < 0).sum() > 100
    host = dst.cpu().numpy()
    for i in np.nonzero(want_res > 0)[0]:
        o = int(doff[i])
        assert np.array_equal(host[o:o + want_res[i]], want_dec[o:o + want_res[i]])


def test_mime(b64, orc, alphs):
    alph, chars, padded = alphs["std"]
    for i, n in enumerate([1, 2, 1000, 1001, 57 * 100 + 1, 300_001]):
        text = orc.encode(wl.random_bytes(n, 80 + i), chars, padded)
        for bit in (0, 1, 2):
            t = spoil_last(text, chars, padded, bit)
            w = wl.mime_wrap(t)
            w = np.concatenate([w, np.frombuffer(b"\r\n \r\n", np.uint8)]) if i % 2 else w
            want_r, want = orc.decode(w, chars, padded, mime=True, canonical=True)
            r, out = b64.mime_decode(torch.from_numpy(w).cuda(), alph)
            assert r == want_r, (n, bit, r, want_r)
            if r >= 0:
                assert np.array_equal(out.cpu().numpy(), want)


def test_host_codec_last_piece(b64, orc, alphs):
    alph, chars, padded = alphs["url"]
    codec = b64.HostCodec(1200, 2)
    try:
        for i, n in enumerate([1, 2, 1000, 900 * 5 + 1, 900 * 5 + 2, 50_001]):
            text = orc.encode(wl.random_bytes(n, 90 + i), chars, padded)
            for bit in (0, 1):
                t = spoil_last(text, chars, padded, bit)
                want_r, _ = orc.decode(t, chars, padded, canonical=True)
                out = np.zeros(b64.decoded_max_length(t.size), np.uint8)
                assert codec.decode(t, out, alph) == want_r, (n, bit)
    finally:
        codec.close()
