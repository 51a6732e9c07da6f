"""Class patterns of 4-character inputs, for the exhaustive 2^32 decode test.

Under the strict rules (Sec. 2 as read: a byte outside the alphabet is an
error at its offset, '=' stands only in the padding positions, the length
rules), the result of decoding a 4-character input depends only on the class
of each byte: 0 = in the alphabet, 1 = '=', 2 = neither. `pattern_table`
takes the oracle's result for one representative string of each of the 81
patterns; tests/test_oracle_quads.py checks the claim on the oracle itself.
"""
import numpy as np

OTHER = 0x21  # '!': in neither alphabet


def byte_classes(chars: bytes) -> np.ndarray:
    cls = np.full(256, 2, np.int64)
    cls[ord("=")] = 1
    cls[np.frombuffer(chars, np.uint8)] = 0
    return cls


def pattern_of(strings: np.ndarray, cls: np.ndarray) -> np.ndarray:
    """strings: (n, 4) uint8 -> pattern ids c0 + 3 c1 + 9 c2 + 27 c3."""
    c = cls[strings]
    return c[:, 0] + 3 * c[:, 1] + 9 * c[:, 2] + 27 * c[:, 3]


def representatives(chars: bytes, pick: int = 0) -> np.ndarray:
    """One string per pattern (81 x 4); `pick` chooses which alphabet
    character stands for class 0."""
    rep = [chars[pick % 64], ord("="), OTHER]
    return np.array([[rep[(p // 3 ** i) % 3] for i in range(4)] for p in range(81)], np.uint8)


def pattern_table(orc, chars: bytes, padded: bool) -> np.ndarray:
    """The oracle's result (length or -(offset+1)) for each of the 81 patterns."""
    s = representatives(chars)
    off = np.arange(82, dtype=np.int64) * 4
    doff = np.arange(82, dtype=np.int64) * 3
    _, res = orc.decode_batch(s.ravel(), off, doff, chars, np.zeros(81, np.int32),
                              np.full(81, int(padded), np.int32), 243)
    return res
