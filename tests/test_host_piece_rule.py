"""The host-buffer codec's piece rule, checked with the oracle on the CPU.

b64_host_decode codes a host buffer in pieces of P characters (P a multiple
of 12): inner pieces are decoded with the padding rule off (every '=' there
is an error, as it is at that position of the whole input), the last piece
always holds the input's last two characters (it is P + 1 characters when
that needs it) and is decoded with the alphabet's own rules, offsets are
shifted by the piece's start, and the first piece with an error gives the
result. b64_host_encode codes pieces of P bytes. The claim is that both give
exactly what the whole-buffer calls give (Sec. 2's padding and length rules
hold for the whole input). Here the rule is applied with the oracle and
compared with the oracle on the whole buffer, over many small pieces and
inputs with errors, '=' and truncations at and around the seams. The GPU
tests run the codec itself.
"""
import numpy as np
import pytest

from paper_1910_05109_gb300 import workloads as wl


def pieces_decode(orc, text, P, chars, padded, canonical):
    m = text.size
    inner = (m - 2) // P if m >= 2 else 0
    out, total = [], 0
    for i in range(inner + 1):
        off = i * P
        n = P if i < inner else m - off
        if i < inner:
            r, o = orc.decode(text[off:off + n], chars, False, canonical=False)
        else:
            r, o = orc.decode(text[off:off + n], chars, padded, canonical=canonical)
        if r < 0:
            return r - off, None
        total += r
        out.append(o[:r])
    return total, np.concatenate(out) if out else np.zeros(0, np.uint8)


def pieces_encode(orc, data, P, chars, padded):
    parts = [orc.encode(data[off:off + P], chars, padded) for off in range(0, data.size, P)]
    return np.concatenate(parts) if parts else np.zeros(0, np.uint8)


TABLES = [("std", True, False), ("url", False, False), ("std", True, True), ("url", False, True)]


@pytest.mark.parametrize("name,padded,canonical", TABLES)
def test_piecewise_decode_equals_whole(orc, name, padded, canonical):
    chars = orc.standard_alphabet() if name == "std" else orc.url_alphabet()
    g = wl.rng(41)
    specials = np.frombuffer(b"=\xff-_+/A\n", np.uint8)
    cases = 0
    for P in (12, 24, 36):
        for trial in range(300):
            n = int(g.integers(0, 8 * P))
            text = orc.encode(wl.random_bytes(n, int(g.integers(1 << 30))), chars, padded)
            text = np.array(text, copy=True)
            kind = trial % 5
            if kind and text.size:
                # edits near a seam, near the end, or anywhere
                for _ in range(int(g.integers(1, 3))):
                    seam = P * int(g.integers(0, text.size // P + 1))
                    at = [seam + int(g.integers(-3, 3)), text.size - 1 - int(g.integers(0, 4)),
                          int(g.integers(0, text.size))][kind % 3]
                    if 0 <= at < text.size:
                        text[at] = specials[int(g.integers(0, specials.size))]
            if kind == 4 and text.size:
                text = text[: text.size - int(g.integers(0, min(5, text.size) + 1))]
            want_r, want = orc.decode(text, chars, padded, canonical=canonical)
            got_r, got = pieces_decode(orc, text, P, chars, padded, canonical)
            assert got_r == want_r, (P, trial, text.tobytes())
            if want_r >= 0:
                assert np.array_equal(got, want[:want_r])
            cases += 1
    assert cases == 900


@pytest.mark.parametrize("name,padded", [("std", True), ("url", False)])
def test_piecewise_encode_equals_whole(orc, name, padded):
    chars = orc.standard_alphabet() if name == "std" else orc.url_alphabet()
    for P in (12, 24, 48):
        for n in list(range(0, 3 * P + 5)) + [10 * P + 1, 10 * P + 2]:
            data = wl.random_bytes(n, 900 + n)
            assert np.array_equal(pieces_encode(orc, data, P, chars, padded),
                                  orc.encode(data, chars, padded)), (P, n)
