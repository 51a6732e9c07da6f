"""Pins of the oracle against what the paper and the mathematics fix.

None of these compare the oracle with itself: each checks it against a value
printed in the paper (Table 1, the Sec. 3.1 worked example, Fig. 2), a library
routine (Python's base64/binascii), an independent model of the paper's SIMD
algorithm (tests/paper_simd_model.py), brute force, or an invariant.
"""
import base64
import binascii
import itertools

import numpy as np
import pytest

from conftest import read_golden
from paper_1910_05109_gb300 import workloads as wl
import paper_simd_model as sm

STD = b"ABCDEFGHIJKLMNOPQRSTUVWXYZabcdefghijklmnopqrstuvwxyz0123456789+/"


def _golden_kv(name):
    return {row[0]: row[1:] for row in read_golden(name)}


# ---------------------------------------------------------------- Table 1

def test_table1_alphabet(orc):
    rows = read_golden("table1.txt")
    assert len(rows) == 64
    alph = orc.standard_alphabet()
    for value, hexcode, ch in rows:
        v, code = int(value), int(hexcode, 16)
        assert ord(ch) == code
        assert alph[v] == code
        assert orc.value_of(alph, code) == v
    members = set(alph)
    for c in range(256):
        if c not in members:
            assert orc.value_of(alph, c) == -1


def test_url_alphabet_substitution(orc):
    # Sec. 2: base64url replaces '+' and '/' by '-' and '_'.
    std, url = orc.standard_alphabet(), orc.url_alphabet()
    assert url[:62] == std[:62]
    assert url[62:] == b"-_" and std[62:] == b"+/"


# ---------------------------------------------------------------- encode

@pytest.mark.parametrize("padded", [True, False])
@pytest.mark.parametrize("url", [False, True])
def test_encode_matches_python_base64(orc, padded, url):
    alph = orc.url_alphabet() if url else orc.standard_alphabet()
    lib = base64.urlsafe_b64encode if url else base64.b64encode
    sizes = list(range(0, 200)) + [1000, 4095, 4096, 4097, 65537, 1 << 20]
    for i, n in enumerate(sizes):
        data = wl.random_bytes(n, seed=100 + i)
        want = lib(data.tobytes())
        if not padded:
            want = want.rstrip(b"=")
        got = orc.encode(data, alph, padded).tobytes()
        assert got == want, n
        assert len(got) == orc.encoded_length(n, padded)


def test_encode_all_triples_and_roundtrip(orc):
    # Brute force over all 2^24 three-byte inputs, concatenated.
    v = np.arange(1 << 24, dtype=np.uint32)
    data = np.stack([(v >> 16) & 255, (v >> 8) & 255, v & 255], axis=1).astype(np.uint8).ravel()
    enc = orc.encode(data)
    assert enc.tobytes() == base64.b64encode(data.tobytes())
    r, dec = orc.decode(enc)
    assert r == data.size
    assert np.array_equal(dec, data)


def test_all_tails(orc):
    # Every 1-byte and 2-byte input (padding cases of Sec. 2), padded and not.
    for n in (1, 2):
        for t in itertools.product(range(256), repeat=n):
            b = bytes(t)
            e = orc.encode(b).tobytes()
            assert e == base64.b64encode(b)
            assert orc.encode(b, padded=False).tobytes() == e.rstrip(b"=")
            r, d = orc.decode(e)
            assert r == n and d.tobytes() == b
            r, d = orc.decode(e.rstrip(b"="), padded=False)
            assert r == n and d.tobytes() == b


def test_encoded_length_closed_form(orc):
    for n in range(0, 1000):
        assert orc.encoded_length(n, True) == 4 * ((n + 2) // 3)
        assert orc.encoded_length(n, False) == (4 * n + 2) // 3


def test_sec31_gather_example_and_block_model(orc):
    g = _golden_kv("encode_gather_shifts.txt")
    rows = [r[1:] for r in read_golden("encode_gather_shifts.txt") if r[0] == "gather"]
    printed = np.array([int(x) for r in rows for x in r])
    # The printed table is what the rule (s1,s2,s3) -> (s2,s1,s3,s2) gives on
    # the byte values 0..63.
    rule = np.array([[3 * t + 1, 3 * t, 3 * t + 2, 3 * t + 1] for t in range(16)]).ravel()
    assert np.array_equal(printed, rule)
    shifts = np.array([int(x) for x in g["shifts"]])
    assert list(shifts[4:]) == [s + 32 for s in shifts[:4]]
    # The paper's three-instruction block encoder (modelled) agrees with the
    # oracle's scalar formulas on random 48-byte blocks, for two alphabets.
    blocks = wl.random_bytes(48 * 4096, seed=7).reshape(4096, 48)
    for alph in (orc.standard_alphabet(), orc.url_alphabet()):
        got = sm.encode_block(blocks, alph, printed, shifts.astype(np.uint8))
        want = orc.encode(blocks.ravel(), alph).reshape(4096, 64)
        assert np.array_equal(got, want)


# ---------------------------------------------------------------- decode

def test_fig2_worked_example(orc):
    g = _golden_kv("fig2_decode.txt")
    inp = np.array([int(x, 16) for x in g["input"]], np.uint8)
    translated = np.array([int(x, 16) for x in g["translated"]], np.uint8)
    msb = np.array([int(x) for x in g["error_msb"]])
    t = sm.decode_translation_table(orc.standard_alphabet())
    x = sm.vpermi2b(inp, t[:64], t[64:])
    assert np.array_equal(x, translated)
    err = sm.ternary_or(np.zeros(4, np.uint8), inp, x)
    assert np.array_equal(err >> 7, msb)
    r, _ = orc.decode(inp)
    assert r == -(int(g["first_bad_offset"][0]) + 1)


def test_decode_block_model_and_garbled_constants(orc):
    """The paper's five-instruction decoder (modelled) reproduces the oracle
    with the multiply-add constant (2^6, 1) and the pack order (2,1,0, 6,5,4,
    ...) derived from the 24-bit layout; the constant (0, 2^6) and the index
    list as printed do not (readings i and ii)."""
    g = _golden_kv("encode_gather_shifts.txt")
    n = 2048
    data = wl.random_bytes(48 * n, seed=8)
    chars = orc.encode(data).reshape(n, 64)
    corrected = np.array([4 * j + k for j in range(16) for k in (2, 1, 0)])
    printed = np.array([int(x) for x in g["pack_printed"]])
    assert len(printed) == 48
    assert sorted(printed) == sorted(corrected)  # same set, different order
    madd2 = tuple(int(x) for x in g["maddwd_printed"])
    assert madd2 == (4096, 1)
    out, err = sm.decode_block(chars, orc.standard_alphabet(), (64, 1), madd2, corrected)
    assert np.array_equal(out.reshape(-1), data)
    assert not (err & 0x80).any()
    bad1, _ = sm.decode_block(chars, orc.standard_alphabet(),
                              tuple(int(x) for x in g["maddubsw_printed"]), madd2, corrected)
    assert not np.array_equal(bad1.reshape(-1), data)
    bad2, _ = sm.decode_block(chars, orc.standard_alphabet(), (64, 1), madd2, printed)
    assert not np.array_equal(bad2.reshape(-1), data)


def test_decode_block_model_error_register(orc):
    # Every byte value, placed anywhere in a valid 64-char block: the modelled
    # error register flags exactly the bytes outside the alphabet, and the
    # oracle reports the first of them.
    alph = orc.standard_alphabet()
    base = orc.encode(wl.random_bytes(48, seed=9))
    members = set(alph)
    for v in range(256):
        for p in (0, 1, 2, 3, 17, 63):
            blk = base.copy()
            blk[p] = v
            _, err = sm.decode_block(blk[None], alph, (64, 1), (4096, 1),
                                     np.array([4 * j + k for j in range(16) for k in (2, 1, 0)]))
            flagged = np.nonzero(err[0] >> 7)[0]
            r, _ = orc.decode(blk)
            if v in members:
                assert flagged.size == 0 and r == 48
            else:
                assert list(flagged) == [p]
                if v == ord("=") and p == 63:
                    # The block model has no padding rule; as the last
                    # character '=' is padding (one byte fewer).
                    assert r == 47
                else:
                    assert r == -(p + 1)


def test_strict_readings_fixture(orc):
    modes = {"padded": (True, False), "unpadded": (False, False), "mime": (True, True)}
    for mode, hexin, result, hexout in read_golden("strict_readings.txt"):
        padded, mime = modes[mode]
        src = b"" if hexin == "-" else bytes.fromhex(hexin)
        r, out = orc.decode(src, padded=padded, mime=mime)
        assert r == int(result), (mode, hexin)
        if r >= 0:
            assert out.tobytes() == (b"" if hexout == "-" else bytes.fromhex(hexout))


def _python_strict(b):
    try:
        return binascii.a2b_base64(b, strict_mode=True)
    except binascii.Error:
        return None


def _stray_pad_after_full_groups(s: bytes) -> bool:
    """Complete 4-character groups followed only by '=' characters. Python's
    strict decoder ignores such padding; reading R2 rejects it (the length is
    not a multiple of 4, or a '=' stands outside the last two places)."""
    body = s.rstrip(b"=")
    return len(body) % 4 == 0 and len(body) > 0 and len(s) > len(body) and b"=" not in body


def _check_against_python(orc, s):
    r, out = orc.decode(s)
    py = _python_strict(s)
    if py is None:
        assert r < 0, s
    elif _stray_pad_after_full_groups(s):
        assert r < 0, s
    else:
        assert r == len(py) and out.tobytes() == py, s


def test_accept_reject_agrees_with_python_strict(orc):
    # Brute force over short strings from a small character set that has
    # alphabet characters, '=', other-alphabet characters, whitespace and
    # high-bit bytes: accept/reject and the decoded bytes agree with Python's
    # strict decoder (which gives no offsets), except for the one documented
    # class where Python is more lenient.
    charset = [b"Q", b"U", b"+", b"=", b"-", b" ", b"\xc3"]
    for k in range(0, 6):
        for t in itertools.product(charset, repeat=k):
            _check_against_python(orc, b"".join(t))
    for k in range(6, 10):
        for t in itertools.product([b"Q", b"=", b"-"], repeat=k):
            _check_against_python(orc, b"".join(t))
    assert _python_strict(b"QQQQ=") is not None and orc.decode(b"QQQQ=")[0] == -6


def test_python_strict_random_mutations(orc):
    g = wl.rng(10)
    for i in range(3000):
        n = int(g.integers(0, 40))
        enc = bytearray(orc.encode(wl.random_bytes(n, 1000 + i)).tobytes())
        for _ in range(int(g.integers(0, 3))):
            if enc:
                enc[int(g.integers(0, len(enc)))] = int(g.integers(0, 256))
        if g.random() < 0.2 and enc:
            del enc[int(g.integers(0, len(enc)))]
        _check_against_python(orc, bytes(enc))


def test_every_invalid_byte_rejected_at_its_offset(orc):
    alph = orc.standard_alphabet()
    bad = wl.invalid_byte_values(alph)
    assert bad.size == 191
    base = orc.encode(wl.random_bytes(30, seed=11))  # 40 chars, no padding
    for v in bad:
        for p in range(base.size):
            s = base.copy()
            s[p] = v
            assert orc.decode(s)[0] == -(p + 1)
    for p in range(base.size - 2):  # '=' outside the padding zone
        s = base.copy()
        s[p] = ord("=")
        assert orc.decode(s)[0] == -(p + 1)


def test_other_alphabet_rejected(orc):
    std, url = orc.standard_alphabet(), orc.url_alphabet()
    data = wl.random_bytes(3000, seed=12)
    e_std, e_url = orc.encode(data, std), orc.encode(data, url)
    for text, other in ((e_std, url), (e_url, std)):
        mism = np.nonzero(np.isin(text, np.frombuffer(b"+/-_", np.uint8)))[0]
        assert mism.size > 0
        assert orc.decode(text, other)[0] == -(int(mism[0]) + 1)


@pytest.mark.parametrize("padded", [True, False])
def test_roundtrip_and_lengths(orc, padded):
    for i, n in enumerate(list(range(0, 120)) + [999, 1000, 1001, 12345]):
        data = wl.random_bytes(n, seed=200 + i)
        for alph in (orc.standard_alphabet(), orc.url_alphabet()):
            e = orc.encode(data, alph, padded)
            r, d = orc.decode(e, alph, padded)
            assert r == n and np.array_equal(d, data)
            m = e.size
            pads = int((e[-2:] == ord("=")).sum()) if m else 0
            if padded:
                assert r == 3 * (m // 4) - pads
            else:
                assert m % 4 != 1


# ---------------------------------------------------------------- MIME mode

def test_mime_matches_python_nonstrict(orc):
    for i, n in enumerate([0, 1, 2, 3, 57, 58, 1000, 100_000]):
        data = wl.random_bytes(n, seed=300 + i)
        wrapped = wl.mime_wrap(orc.encode(data))
        # Python's non-strict decoder skips every non-alphabet byte; on input
        # whose only extra bytes are CR/LF it must agree with MIME mode.
        want = binascii.a2b_base64(wrapped.tobytes())
        r, out = orc.decode(wrapped, mime=True)
        assert r == n and out.tobytes() == want == data.tobytes()
        # Python's own MIME encoder (76-char lines) decodes the same way.
        r2, out2 = orc.decode(np.frombuffer(base64.encodebytes(data.tobytes()), np.uint8),
                              mime=True)
        assert r2 == n and out2.tobytes() == data.tobytes()


def test_mime_whitespace_everywhere_brute(orc):
    # Inserting CR, LF or SP anywhere changes nothing but the coordinates of
    # an error: an error at compacted index j is reported at the original
    # index of that character, a length error at the original length.
    cases = [b"QUJD", b"QQ==", b"QUI=", b"QQ=A", b"Q===", b"QU\xc3D", b"Q", b"QQ="]
    for s in cases:
        r0, out0 = orc.decode(s)
        for p in range(len(s) + 1):
            for w in (b"\r", b"\n", b" ", b"\r\n"):
                t = s[:p] + w + s[p:]
                r, out = orc.decode(t, mime=True)
                if r0 >= 0:
                    assert r == r0 and out.tobytes() == out0.tobytes()
                else:
                    off = -r0 - 1
                    if off == len(s):
                        want = len(t)
                    else:
                        want = off + (len(w) if off >= p else 0)
                    assert r == -(want + 1), (s, p, w)
        # Outside MIME mode the same whitespace is an error at its index.
        if len(s) >= 2:
            t = s[:1] + b"\n" + s[1:]
            r, _ = orc.decode(t)
            assert r == -2 or (r0 < 0 and r == -(min(-r0 - 1, 1) + 1))


def test_tab_is_not_mime_space(orc):
    assert orc.decode(b"QQ\t==", mime=True)[0] == -3


# ---------------------------------------------------------------- batched loops

def test_batch_equals_single_calls(orc):
    std, url = orc.standard_alphabet(), orc.url_alphabet()
    data, off = wl.varlen_strings(300, seed=13, median=64, sigma=1.5, hi=4096)
    n = off.size - 1
    alph_id = wl.bernoulli(n, 14)
    padded = 1 - alph_id
    elen = np.array([orc.encoded_length(int(off[i + 1] - off[i]), bool(padded[i]))
                     for i in range(n)])
    doff = wl.offsets_from_lengths(elen)
    enc, res = orc.encode_batch(data, off, doff, std + url, alph_id, padded, int(doff[-1]))
    for i in range(n):
        a = url if alph_id[i] else std
        want = orc.encode(data[off[i]:off[i + 1]], a, bool(padded[i]))
        assert res[i] == want.size
        assert np.array_equal(enc[doff[i]:doff[i + 1]], want)
    dlen = off[1:] - off[:-1]
    dec, dres = orc.decode_batch(enc, doff, off, std + url, alph_id, padded, int(off[-1]))
    assert np.array_equal(dres, dlen)
    assert np.array_equal(dec, data)
