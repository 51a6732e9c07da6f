"""Word-parallel whitespace tests of the MIME count kernel, checked on the CPU.

The kernel marks the bytes of a 32-bit word equal to a byte c without
comparing them one by one: with t = x ^ (c * 0x01010101),
~(((t & 0x7F7F7F7F) + 0x7F7F7F7F) | t) & 0x80808080 has bit 7 of a byte set
exactly when that byte of t is zero. A carry could only pass from one byte to
the next higher one, so checking every pair of adjacent bytes (all 65,536
values, in each of the three positions) proves the test exact for whole
words. The counts and the last data byte of a 16-byte chunk built on it are
compared with their direct definitions on random chunks rich in CR, LF and
space. The kernel's formulas are restated with numpy.
"""
import numpy as np

M7F, M80 = np.uint32(0x7F7F7F7F), np.uint32(0x80808080)


def eq_bytes(x, c):
    t = x ^ np.uint32(c * 0x01010101)
    return ~(((t & M7F) + M7F) | t) & M80


def space_bytes(x):
    return eq_bytes(x, 0x0D) | eq_bytes(x, 0x0A) | eq_bytes(x, 0x20)


def test_byte_equality_is_exact_for_every_adjacent_pair():
    pair = np.arange(1 << 16, dtype=np.uint32)
    g = np.random.default_rng(3)
    for shift in (0, 8, 16):
        rest = g.integers(0, 1 << 32, pair.size, dtype=np.uint64).astype(np.uint32)
        keep = ~np.uint32(0xFFFF << shift)
        x = (rest & keep) | (pair << np.uint32(shift))
        for c in (0x0D, 0x0A, 0x20, 0x00, 0x80, 0xFF, 0x7F):
            got = eq_bytes(x, c)
            for k in range(4):
                byte = (x >> np.uint32(8 * k)) & np.uint32(0xFF)
                bit = (got >> np.uint32(8 * k + 7)) & np.uint32(1)
                assert np.array_equal(bit == 1, byte == c), (shift, c, k)
            assert not np.any(got & ~M80)


def chunk_data(words):
    return sum(bin(int(~space_bytes(w) & M80)).count("1") for w in words)


def chunk_last(words, off):
    d = [int(~space_bytes(w) & M80) for w in words]
    hi = 0xFF
    for j in (3, 2, 1, 0):
        if d[j]:
            hi = 4 * j + (d[j].bit_length() - 1) // 8
            break
    if hi == 0xFF:
        return 0
    b = (int(words[hi // 4]) >> (8 * (hi % 4))) & 0xFF
    return ((off + hi + 1) << 8) | b


def test_chunk_count_and_last_data_byte():
    g = np.random.default_rng(5)
    pool = np.frombuffer(b"\r\n  \r\n ABz+/=\x00\xff\x09", np.uint8)
    for trial in range(20_000):
        chunk = pool[g.integers(0, pool.size, 16)] if trial % 3 else \
            np.frombuffer(b"\r\n" * 8, np.uint8).copy()
        if trial % 7 == 0:
            chunk[g.integers(0, 16)] = g.integers(0, 256)
        words = chunk.view("<u4").astype(np.uint32)
        data = [i for i in range(16) if chunk[i] not in (0x0D, 0x0A, 0x20)]
        assert chunk_data(words) == len(data)
        off = int(g.integers(0, 4096 - 16)) // 16 * 16
        want = ((off + data[-1] + 1) << 8) | int(chunk[data[-1]]) if data else 0
        assert chunk_last(words, off) == want
