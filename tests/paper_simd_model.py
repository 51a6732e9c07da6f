"""numpy model of the AVX-512 instruction semantics the paper describes.

Sec. 3.1 and Sec. 3.2 describe each instruction in words; these functions
restate those descriptions over numpy arrays of 64-byte registers (shape
[..., 64], byte 0 = least significant / lowest address). Tests run the
paper's block algorithms through this model and compare the result with the
oracle, which computes the same thing from the scalar formulas of Sec. 2.
Two independent routes to one result pin both.
"""
from __future__ import annotations

import numpy as np


def vpermb(idx: np.ndarray, table: np.ndarray) -> np.ndarray:
    """out[i] = table[idx[i]], only the six low bits of each index used (Sec. 3.1)."""
    return np.take_along_axis(table, (idx & 63).astype(np.int64), axis=-1)


def vpmultishiftqb(shifts: np.ndarray, data: np.ndarray) -> np.ndarray:
    """For each 64-bit word of ``data`` and each of its eight shift bytes: rotate
    the word right by (shift mod 64) and keep the low eight bits (Sec. 3.1)."""
    words = data.reshape(*data.shape[:-1], 8, 8).astype(np.uint64)
    w = np.zeros(words.shape[:-1], np.uint64)
    for k in range(8):
        w |= words[..., k] << np.uint64(8 * k)
    sh = (shifts.reshape(*shifts.shape[:-1], 8, 8) & 63).astype(np.uint64)
    w = w[..., None]
    rot = (w >> sh) | np.where(sh == 0, np.uint64(0), w << ((np.uint64(64) - sh) & np.uint64(63)))
    return (rot & np.uint64(0xFF)).astype(np.uint8).reshape(data.shape)


def vpermi2b(idx: np.ndarray, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """128-entry lookup in the concatenation of a and b; the top bit of each
    index is ignored (Sec. 3.2)."""
    table = np.concatenate([a, b], axis=-1)
    return np.take_along_axis(table, (idx & 127).astype(np.int64), axis=-1)


def ternary_or(x: np.ndarray, y: np.ndarray, z: np.ndarray) -> np.ndarray:
    """vpternlogd configured as x OR y OR z (Sec. 3.2)."""
    return x | y | z


def vpmovb2m(x: np.ndarray) -> np.ndarray:
    """64-bit mask of the most significant bits of the 64 bytes (Sec. 3.2)."""
    bits = (x >> 7).astype(np.uint64)
    return (bits << np.arange(64, dtype=np.uint64)).sum(axis=-1, dtype=np.uint64)


def vpmaddubsw(u: np.ndarray, s: np.ndarray) -> np.ndarray:
    """Per 16-bit block: unsigned bytes of ``u`` times signed bytes of ``s``,
    the two products added (Sec. 3.2). Returns int32 values per block."""
    uu = u.astype(np.int32).reshape(*u.shape[:-1], -1, 2)
    ss = s.astype(np.int8).astype(np.int32).reshape(*s.shape[:-1], -1, 2)
    r = (uu * ss).sum(axis=-1)
    return np.clip(r, -32768, 32767)


def vpmaddwd(x16: np.ndarray, c16: np.ndarray) -> np.ndarray:
    """Per 32-bit block: the two signed 16-bit values times the constant's two
    16-bit values, added (Sec. 3.2)."""
    xx = x16.astype(np.int64).reshape(*x16.shape[:-1], -1, 2)
    cc = c16.astype(np.int64).reshape(*c16.shape[:-1], -1, 2)
    return (xx * cc).sum(axis=-1)


def words_to_bytes(w32: np.ndarray) -> np.ndarray:
    w = w32.astype(np.uint32)
    return np.stack([(w >> (8 * k)) & 0xFF for k in range(4)], axis=-1).astype(np.uint8).reshape(
        *w.shape[:-1], -1)


def encode_block(block48: np.ndarray, alphabet: bytes, gather: np.ndarray,
                 shifts: np.ndarray) -> np.ndarray:
    """Sec. 3.1: 48 input bytes (in a 64-byte register) -> 64 characters with
    vpermb (gather), vpmultishiftqb (shifts), vpermb (alphabet)."""
    reg = np.zeros((*block48.shape[:-1], 64), np.uint8)
    reg[..., :48] = block48
    g = vpermb(np.broadcast_to(gather, reg.shape), reg)
    sh = vpmultishiftqb(np.broadcast_to(np.tile(shifts, 8), reg.shape).astype(np.uint8), g)
    table = np.broadcast_to(np.frombuffer(alphabet, np.uint8), reg.shape)
    return vpermb(sh, table)


def decode_translation_table(alphabet: bytes) -> np.ndarray:
    """Sec. 3.2: 128 entries, 0x80 everywhere except at the alphabet's code
    points, which hold their 6-bit values."""
    t = np.full(128, 0x80, np.uint8)
    for k, c in enumerate(alphabet):
        t[c] = k
    return t


def decode_block(chars64: np.ndarray, alphabet: bytes, madd1: tuple[int, int],
                 madd2: tuple[int, int], pack_idx: np.ndarray):
    """Sec. 3.2: 64 characters -> (48 bytes, error register) with vpermi2b,
    vpternlogd, vpmaddubsw, vpmaddwd and vpermb."""
    t = decode_translation_table(alphabet)
    x = vpermi2b(chars64, np.broadcast_to(t[:64], chars64.shape),
                 np.broadcast_to(t[64:], chars64.shape))
    err = ternary_or(np.zeros_like(chars64), chars64, x)
    c1 = np.broadcast_to(np.tile(np.array(madd1, np.int64), 32), chars64.shape)
    m1 = vpmaddubsw(x, c1.astype(np.int8))
    c2 = np.broadcast_to(np.tile(np.array(madd2, np.int64), 16), m1.shape)
    m2 = vpmaddwd(m1, c2)
    reg = words_to_bytes(m2.astype(np.int64) & 0xFFFFFFFF)
    full = np.zeros((*chars64.shape[:-1], 64), np.int64)
    full[..., :48] = pack_idx
    out = vpermb(full, reg)[..., :48]
    return out, err
