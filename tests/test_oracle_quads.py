"""Pins for the class-pattern table used by the exhaustive 4-byte GPU test.

- The oracle's result on any 4-byte input equals the table entry of its
  class pattern (random inputs, and every pattern with other representatives).
- Counting the 2^32 inputs by pattern gives the closed forms of Sec. 2's
  rules: 64^4 + 64^3 + 64^2 valid padded inputs (3, 2 and 1 bytes), 64^4
  valid unpadded ones, and 192 * 256^3 inputs failing at offset 0 (a first
  byte that is '=' or outside the alphabet).
"""
import numpy as np
import pytest

import quad_classes as qc
from paper_1910_05109_gb300 import workloads as wl

MODES = [("std", True), ("url", False)]


def chars_of(orc, name):
    return orc.standard_alphabet() if name == "std" else orc.url_alphabet()


@pytest.mark.parametrize("name,padded", MODES)
def test_result_depends_only_on_class_pattern(orc, name, padded):
    chars = chars_of(orc, name)
    table = qc.pattern_table(orc, chars, padded)
    cls = qc.byte_classes(chars)
    g = wl.rng(40)
    # random bytes, and random draws from {alphabet, '=', other} so that
    # every pattern is well represented
    pools = [np.frombuffer(chars, np.uint8), np.array([ord("=")], np.uint8),
             np.array([b for b in range(256) if cls[b] == 2], np.uint8)]
    n = 400_000
    s1 = g.integers(0, 256, (n, 4)).astype(np.uint8)
    which = g.integers(0, 3, (n, 4))
    s2 = np.empty((n, 4), np.uint8)
    for k in range(3):
        m = which == k
        s2[m] = pools[k][g.integers(0, pools[k].size, m.sum())]
    s = np.concatenate([s1, s2])
    off = np.arange(s.shape[0] + 1, dtype=np.int64) * 4
    doff = np.arange(s.shape[0] + 1, dtype=np.int64) * 3
    _, res = orc.decode_batch(s.ravel(), off, doff, chars, np.zeros(s.shape[0], np.int32),
                              np.full(s.shape[0], int(padded), np.int32), 3 * s.shape[0])
    assert np.array_equal(res, table[qc.pattern_of(s, cls)])
    for pick in (1, 17, 63):
        r = qc.representatives(chars, pick)
        _, res = orc.decode_batch(r.ravel(), np.arange(82, dtype=np.int64) * 4,
                                  np.arange(82, dtype=np.int64) * 3, chars,
                                  np.zeros(81, np.int32), np.full(81, int(padded), np.int32), 243)
        assert np.array_equal(res, table)


@pytest.mark.parametrize("name,padded", MODES)
def test_pattern_counts_match_closed_forms(orc, name, padded):
    table = qc.pattern_table(orc, chars_of(orc, name), padded)
    size = np.array([64, 1, 191], np.int64)
    count = np.array([size[(p // 1) % 3] * size[(p // 3) % 3] * size[(p // 9) % 3] * size[p // 27]
                      for p in range(81)])
    assert count.sum() == 256 ** 4
    by = lambda r: int(count[table == r].sum())
    if padded:
        assert (by(3), by(2), by(1)) == (64 ** 4, 64 ** 3, 64 ** 2)
        assert int(count[table >= 0].sum()) == 64 ** 4 + 64 ** 3 + 64 ** 2
    else:
        assert by(3) == 64 ** 4 and int(count[table >= 0].sum()) == 64 ** 4
    assert by(-1) == 192 * 256 ** 3
