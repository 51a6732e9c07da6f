"""Property pins of the oracle (no GPU), independent of how it is written:
invariants that Sec. 2's mappings and the strict readings fix for every
input, checked on random inputs.

- Round trip: decode(encode(b)) == b, with the lengths of Sec. 2 (4 ceil(n/3)
  padded, ceil(4n/3) unpadded), for the standard and base64url tables and a
  shuffled custom table.
- What the encoder emits is canonical (R7 accepts it).
- Whitespace (CR, LF, space) inserted anywhere leaves a MIME decode's output
  unchanged (R5).
- One byte outside the alphabet (and not '=') placed before the last four
  characters of a valid encoding is reported at its own offset (R1, R4), also
  in MIME mode with whitespace before it, in original coordinates.
"""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

STD = b"ABCDEFGHIJKLMNOPQRSTUVWXYZabcdefghijklmnopqrstuvwxyz0123456789+/"
URL = STD[:62] + b"-_"
CUSTOM = bytes(np.random.default_rng(5).permutation(np.frombuffer(STD, np.uint8)))
TABLES = [STD, URL, CUSTOM]
WS = [13, 10, 32]

settings.register_profile("oracle", max_examples=300, deadline=None)
settings.load_profile("oracle")


@given(st.binary(max_size=400), st.sampled_from(TABLES), st.booleans())
def test_round_trip_and_lengths(orc, data, chars, padded):
    text = orc.encode(np.frombuffer(data, np.uint8), chars, padded)
    n = len(data)
    assert text.size == ((n + 2) // 3 * 4 if padded else (4 * n + 2) // 3)
    assert set(text.tobytes()) <= set(chars + (b"=" if padded else b""))
    r, out = orc.decode(text, chars, padded)
    assert r == n and out.tobytes() == data
    r, out = orc.decode(text, chars, padded, canonical=True)
    assert r == n and out.tobytes() == data


@given(st.binary(min_size=1, max_size=300), st.sampled_from(TABLES), st.booleans(),
       st.lists(st.tuples(st.integers(0, 10_000), st.sampled_from(WS)), max_size=40))
def test_whitespace_anywhere_changes_nothing(orc, data, chars, padded, inserts):
    text = list(orc.encode(np.frombuffer(data, np.uint8), chars, padded).tobytes())
    for pos, c in inserts:
        text.insert(pos % (len(text) + 1), c)
    r, out = orc.decode(np.array(text, np.uint8), chars, padded, mime=True)
    assert r == len(data) and out.tobytes() == data


@given(st.binary(min_size=6, max_size=300), st.sampled_from(TABLES), st.booleans(),
       st.integers(0, 10_000), st.integers(0, 255), st.integers(0, 30))
def test_one_bad_byte_is_reported_where_it_is(orc, data, chars, padded, pos, bad, spaces):
    text = orc.encode(np.frombuffer(data, np.uint8), chars, padded)
    if bad in chars or bad == ord("=") or bad in WS:
        bad = 0x21  # '!': in none of the tables
    p = pos % (text.size - 4)  # before the last group: no padding rule can fire first
    t = text.copy()
    t[p] = bad
    assert orc.decode(t, chars, padded)[0] == -(p + 1)
    # MIME: spaces in front of it move the offset by their number
    m = np.concatenate([np.full(spaces, 32, np.uint8), t])
    assert orc.decode(m, chars, padded, mime=True)[0] == -(p + spaces + 1)
