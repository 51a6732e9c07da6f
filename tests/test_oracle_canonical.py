"""Pins of the oracle's canonical mode (reading R7: RFC 4648 Sec. 3.5 lets a
decoder reject the non-zero unused bits an encoder never emits).

Checked against Python's own encoder (canonical by construction), Table 1
values computed from the alphabet string, hand-derived cases
(tests/golden/canonical_readings.txt) and a closed-form count over every
four-character string.
"""
import base64
import itertools

import numpy as np

from conftest import read_golden
from paper_1910_05109_gb300 import workloads as wl

STD = b"ABCDEFGHIJKLMNOPQRSTUVWXYZabcdefghijklmnopqrstuvwxyz0123456789+/"
URL = STD[:62] + b"-_"


def unescape(t: str) -> bytes:
    return t.replace("\\r", "\r").replace("\\n", "\n").encode()


def test_fixture(orc):
    for text, padded, want in read_golden("canonical_readings.txt"):
        chars = STD if padded == "1" else URL
        r, _ = orc.decode(unescape(text), chars, padded == "1", canonical=True)
        assert r == int(want), (text, padded, r, want)
        # without the flag only the R3 reading applies (non-canonical accepted)
        r3, _ = orc.decode(unescape(text), chars, padded == "1")
        if int(want) >= 0:
            assert r3 == int(want)


def test_python_encodings_are_canonical(orc):
    # every 0..2-byte input and random longer ones, both tables and modes
    inputs = [bytes(t) for n in (0, 1, 2) for t in itertools.product(range(256), repeat=n)]
    g = wl.rng(61)
    inputs += [g.integers(0, 256, int(g.integers(3, 300)), dtype=np.uint8).tobytes()
               for _ in range(300)]
    for b in inputs:
        for chars, enc in ((STD, base64.b64encode(b)), (URL, base64.urlsafe_b64encode(b))):
            for padded in (True, False):
                e = enc if padded else enc.rstrip(b"=")
                r, d = orc.decode(e, chars, padded, canonical=True)
                assert r == len(b) and d.tobytes() == b


def test_final_groups_closed_form(orc):
    # "AY==": the 4 low bits of Y reach no byte; "AAZ=": the 2 low bits of Z
    for v, c in enumerate(STD):
        r, _ = orc.decode(b"A" + bytes([c]) + b"==", STD, True, canonical=True)
        assert r == (1 if v % 16 == 0 else -2), (chr(c), r)
        r, _ = orc.decode(b"AA" + bytes([c]) + b"=", STD, True, canonical=True)
        assert r == (2 if v % 4 == 0 else -3), (chr(c), r)
        r, _ = orc.decode(b"A" + bytes([c]), URL, False, canonical=True)
        assert r == (1 if v % 16 == 0 else -2)


def test_every_four_character_string_count(orc):
    # over the table plus '=': accepted = 64^4 full groups + 64*4 "XY==" with
    # Y mod 16 = 0 + 64*64*16 "XYZ=" with Z mod 4 = 0
    sym = np.frombuffer(STD + b"=", np.uint8)
    idx = np.arange(65 ** 4)
    strings = np.stack([sym[(idx // 65 ** k) % 65] for k in (3, 2, 1, 0)], axis=1)
    n = strings.shape[0]
    off = np.arange(n + 1, dtype=np.int64) * 4
    _, res = orc.decode_batch(strings.ravel(), off, np.arange(n + 1, dtype=np.int64) * 3, STD,
                              np.zeros(n, np.int32), np.full(n, 3, np.int32), 3 * n)
    assert (res >= 0).sum() == 64 ** 4 + 64 * 4 + 64 * 64 * 16
    # without the flag: every 64*64 "XY==" and 64^3 "XYZ=" are accepted
    _, res3 = orc.decode_batch(strings.ravel(), off, np.arange(n + 1, dtype=np.int64) * 3, STD,
                               np.zeros(n, np.int32), np.full(n, 1, np.int32), 3 * n)
    assert (res3 >= 0).sum() == 64 ** 4 + 64 * 64 + 64 ** 3


def test_mime_offsets_in_original_coordinates(orc):
    # whitespace anywhere moves only the reported offset
    for text, want in ((b"QR\r\n==", -2), (b"Q\r\nR==", -4), (b"QUJD\r\nQUJ=", -9),
                       (b" QUI=\r\n", 2)):
        r, _ = orc.decode(text, STD, True, mime=True, canonical=True)
        assert r == want, (text, r)
