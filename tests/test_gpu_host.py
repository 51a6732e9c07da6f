"""Host-buffer codec (pieces copied in, coded and copied out on several
streams) against the oracle on the whole buffer.

Small pieces (1200 bytes) make every case span many pieces; the decode cases
put '=' and bad bytes at the piece seams, where a piece-by-piece decode that
applied the padding rule to each piece would disagree with the strict reading
of the whole input (Sec. 2: '=' only at the last two positions).
"""
import numpy as np
import pytest
import torch

from paper_1910_05109_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

P = 1200


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
def codecs(b64):
    cs = {s: b64.HostCodec(P, s) for s in (1, 3)}
    yield cs
    for c in cs.values():
        c.close()


def alphabets(b64, orc):
    return [(b64.Alphabet.standard(), orc.standard_alphabet(), True),
            (b64.Alphabet.url(), orc.url_alphabet(), False)]


SIZES = [0, 1, 2, 3, 4, 11, 12, 13, P - 1, P, P + 1, P + 2, 2 * P, 5 * P + 7, 17 * P + 1000]


def host_buf(n, pinned):
    """Page-locked (torch pin_memory) or pageable (numpy) host buffer."""
    if pinned:
        return torch.empty(max(n, 1), dtype=torch.uint8).pin_memory()[:n]
    return np.empty(n, np.uint8)


def as_np(b):
    return b.numpy() if isinstance(b, torch.Tensor) else b


# (input pinned, output pinned): page-locked, pageable and mixed pairs
@pytest.mark.parametrize("pinned", [(True, True), (False, False), (True, False), (False, True)])
def test_host_roundtrip_sizes(b64, orc, codecs, pinned):
    pin_in, pin_out = pinned
    for streams, codec in codecs.items():
        for k, (a, chars, padded) in enumerate(alphabets(b64, orc)):
            for n in SIZES:
                data = wl.random_bytes(n, 100 + n + k)
                src = host_buf(n, pin_in)
                as_np(src)[:] = data
                want = orc.encode(data, chars, padded)
                txt = host_buf(want.size, pin_out)
                assert codec.encode(src, txt, a) == want.size
                assert np.array_equal(as_np(txt), want), (streams, n)
                out = host_buf(b64.decoded_max_length(want.size), pin_in)
                assert codec.decode(txt, out, a) == n
                assert np.array_equal(as_np(out)[:n], data), (streams, n)


def seam_cases():
    """(length, {position: byte}) pairs: '=' and bad bytes at piece edges."""
    eq, bad = ord("="), 0x2A  # '*' is outside both alphabets
    cases = []
    for m in (P + 1, P + 2, P + 3, P + 4, 2 * P, 2 * P + 1, 2 * P + 2, 2 * P + 3, 3 * P + 4):
        cases += [
            (m, {m - 1: eq}), (m, {m - 1: eq, m - 2: eq}), (m, {m - 2: eq}),
            (m, {m - 3: eq, m - 2: eq, m - 1: eq}),
            (m, {P - 1: eq}), (m, {P - 2: eq, P - 1: eq}), (m, {P: eq}),
            (m, {P - 1: bad}), (m, {P: bad}), (m, {P - 1: bad, m - 1: eq}),
            (m, {P + 1: bad, P - 3: eq}), (m, {m - 1: bad}),
        ]
    return cases


def test_host_decode_seams_strict(b64, orc, codecs):
    g = wl.rng(7)
    checked = errors = 0
    for streams, codec in codecs.items():
        for a, chars, padded in alphabets(b64, orc):
            table = np.frombuffer(chars, np.uint8)
            for m, edits in seam_cases():
                text = table[g.integers(0, 64, m)].copy()
                for p, v in edits.items():
                    if 0 <= p < m:
                        text[p] = v
                want_r, want_b = orc.decode(text, chars, padded)
                src = host_buf(m, True)
                src.numpy()[:] = text
                out = host_buf(b64.decoded_max_length(m), True)
                r = codec.decode(src, out, a)
                assert r == want_r, (streams, padded, m, edits, r, want_r)
                if r >= 0:
                    assert np.array_equal(out.numpy()[:r], want_b)
                checked += 1
                errors += r < 0
    assert checked == 2 * 2 * len(seam_cases()) and errors > checked // 2


@pytest.mark.parametrize("pinned", [True, False])
def test_host_large_default_piece(b64, orc, pinned):
    """64 MiB + 5 bytes with the default pieces and streams, one bad byte in
    the decode input at a seeded offset past the first piece; page-locked
    and pageable buffers."""
    n = (64 << 20) + 5
    codec = b64.HostCodec()
    try:
        assert codec.device_bytes() > 0
        data = wl.random_bytes(n, 3)
        src = host_buf(n, pinned)
        as_np(src)[:] = data
        m = b64.encoded_length(n, True)
        txt = host_buf(m, pinned)
        assert codec.encode(src, txt) == m
        want = orc.encode(data)
        assert np.array_equal(as_np(txt), want)
        out = host_buf(b64.decoded_max_length(m), pinned)
        for _ in range(2):  # a second call on the same codec
            as_np(out)[:] = 0
            assert codec.decode(txt, out) == n
            assert np.array_equal(as_np(out)[:n], data)
        g = wl.rng(4)
        pos = int(g.integers(50 << 20, m - 8))
        as_np(txt)[pos] = 0xC3
        r = codec.decode(txt, out)
        assert r == -(pos + 1) == orc.decode(as_np(txt))[0]
    finally:
        codec.close()


def test_host_argument_errors(b64):
    codec = b64.HostCodec(P, 2)
    try:
        with pytest.raises(ValueError):
            codec.encode(np.zeros(10, np.uint8), np.zeros(4, np.uint8))
        with pytest.raises(ValueError):
            codec.decode(np.zeros(8, np.uint8), np.zeros(2, np.uint8))
    finally:
        codec.close()
    with pytest.raises(b64.B64Error):
        b64.HostCodec(P, 9)
