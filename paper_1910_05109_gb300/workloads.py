"""Seeded synthetic inputs for tests, the benchmark and the serving demo.

This module draws random numbers and lays bytes out; it holds none of the
codec's arithmetic, so both the oracle side and the GPU side of a parity test
can take their inputs from it. All generators use numpy's PCG64 with an
explicit seed.

The paper measures on random bytes (Sec. 4, Fig. 4) and states that the
vectorised codecs are insensitive to content (Sec. 4, Table 2); its image and
zip files are not available, so uniform random bytes stand in for them, at
the paper's own sizes where a test wants them.
"""
from __future__ import annotations

import numpy as np

# File sizes of Table 2 (Sec. 4): lena, mandril, Google logo, large zip.
TABLE2_SIZES = (141_020, 247_222, 2_357, 34_904_444)

# Characters removed before decoding in MIME mode.
MIME_SPACE = b"\r\n "


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def random_bytes(n: int, seed: int) -> np.ndarray:
    """n uniform random bytes."""
    return rng(seed).integers(0, 256, size=n, dtype=np.uint8)


def invalid_byte_values(alphabet: bytes, allowed_extra: bytes = b"=") -> np.ndarray:
    """All byte values that are neither in ``alphabet`` nor in ``allowed_extra``."""
    taken = np.zeros(256, bool)
    taken[np.frombuffer(alphabet + allowed_extra, np.uint8)] = True
    return np.nonzero(~taken)[0].astype(np.uint8)


def inject_invalid(chars: np.ndarray, seed: int, alphabet: bytes,
                   allowed_extra: bytes = b"=") -> tuple[np.ndarray, int, int]:
    """Copy of ``chars`` with one byte replaced, at an offset drawn uniformly
    from [0, len), by a value drawn uniformly from the bytes outside the
    alphabet and ``allowed_extra``. Returns (copy, offset, value)."""
    g = rng(seed)
    out = np.array(chars, dtype=np.uint8, copy=True)
    if out.size == 0:
        return out, -1, -1
    off = int(g.integers(0, out.size))
    bad = invalid_byte_values(alphabet, allowed_extra)
    val = int(bad[g.integers(0, bad.size)])
    out[off] = val
    return out, off, val


def lognormal_lengths(count: int, seed: int, median: float, sigma: float,
                      lo: int, hi: int) -> np.ndarray:
    """``count`` lengths from a lognormal with the given median and sigma,
    rounded and clipped to [lo, hi]."""
    x = rng(seed).lognormal(mean=np.log(median), sigma=sigma, size=count)
    return np.clip(np.rint(x), lo, hi).astype(np.int64)


def offsets_from_lengths(lengths: np.ndarray) -> np.ndarray:
    off = np.zeros(len(lengths) + 1, np.int64)
    np.cumsum(lengths, out=off[1:])
    return off


def varlen_strings(count: int, seed: int, median: int = 1024, sigma: float = 1.5,
                   lo: int = 1, hi: int = 1 << 20) -> tuple[np.ndarray, np.ndarray]:
    """Concatenated random strings with lognormal lengths. Returns
    (bytes, offsets[count+1])."""
    lengths = lognormal_lengths(count, seed, median, sigma, lo, hi)
    off = offsets_from_lengths(lengths)
    data = random_bytes(int(off[-1]), seed + 1_000_003)
    return data, off


def bernoulli(count: int, seed: int, p: float = 0.5) -> np.ndarray:
    return (rng(seed).random(count) < p).astype(np.int32)


def mime_wrap(chars: np.ndarray, line: int = 76, eol: bytes = b"\r\n") -> np.ndarray:
    """Inserts ``eol`` after every ``line`` characters, except after the last
    line (no trailing line break)."""
    chars = np.asarray(chars, np.uint8)
    n = chars.size
    if n == 0:
        return chars.copy()
    nlines = (n + line - 1) // line
    e = np.frombuffer(eol, np.uint8)
    out = np.empty(n + (nlines - 1) * e.size, np.uint8)
    full = n // line if n % line else nlines - 1
    stride = line + e.size
    if full:
        body = out[: full * stride].reshape(full, stride)
        body[:, :line] = chars[: full * line].reshape(full, line)
        body[:, line:] = e
    rest = chars[full * line:]
    out[full * stride:] = rest
    return out


def insert_spaces(chars: np.ndarray, seed: int, count: int,
                  choices: bytes = MIME_SPACE) -> np.ndarray:
    """Inserts ``count`` characters drawn from ``choices`` at random positions."""
    g = rng(seed)
    chars = np.asarray(chars, np.uint8)
    pos = np.sort(g.integers(0, chars.size + 1, size=count))
    vals = np.frombuffer(choices, np.uint8)[g.integers(0, len(choices), size=count)]
    return np.insert(chars, pos, vals)


def poisson_arrivals(rate_hz: float, duration_s: float, seed: int) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process over [0, duration)."""
    g = rng(seed)
    n_guess = int(rate_hz * duration_s * 1.2 + 100)
    t = np.cumsum(g.exponential(1.0 / rate_hz, size=n_guess))
    while t[-1] < duration_s:
        more = t[-1] + np.cumsum(g.exponential(1.0 / rate_hz, size=n_guess))
        t = np.concatenate([t, more])
    return t[t < duration_s]
