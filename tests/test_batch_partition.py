"""How the batched kernels split work between warps, checked on the CPU.

The concatenated input [src_off[0], src_off[n]) is cut into GW equal byte
ranges, one per warp. Each range end x is moved to the next 3-byte (encode)
or 4-character (decode) group boundary of the string holding x, found by a
32-way search over src_off in which every lane probes one of 32 evenly
spaced candidates and a ballot keeps the last that is <= x, but not past the
end of the string's coded part (encode: the whole string; decode: all but
its last 2..5 characters, which the finalize kernel decodes). Each warp then
walks its range string by string in tiles of at most T bytes. Restated here
in Python and run over batches with empty, tiny and long strings and warp
counts from 1 to more warps than groups: the tiles of all warps must cover
every string's coded part exactly once, each tile inside one string and
starting on one of its group boundaries. The GPU tests run the kernels on
the same kinds of batches.
"""
import bisect

import numpy as np
import pytest


def body_length(m):
    return (m - 2) & ~3 if m >= 2 else 0


def warp_find_string(src_off, n, x):
    lo, hi = 0, n
    while hi - lo > 1:
        step = (hi - lo + 31) // 32
        mask = 0
        for lane in range(32):
            probe = lo + lane * step
            if probe < hi and src_off[probe] <= x:
                mask |= 1 << lane
        k = mask.bit_length() - 1
        nlo = lo + k * step
        lo, hi = nlo, min(nlo + step, hi)
    return lo


def round_boundary(src_off, n, x, decode):
    if x >= src_off[n]:
        return src_off[n]
    s = warp_find_string(src_off, n, x)
    s0, ln = src_off[s], src_off[s + 1] - src_off[s]
    lim = body_length(ln) if decode else ln
    g = 4 if decode else 3
    r = (x - s0 + g - 1) // g * g
    return s0 + min(r, lim)


def warp_tiles(src_off, n, gw, GW, T, decode):
    origin, total = src_off[0], src_off[n] - src_off[0]
    if total <= 0:
        return []
    x0 = origin + total * gw // GW
    x1 = origin + total * (gw + 1) // GW
    pos = round_boundary(src_off, n, x0, decode)
    end = src_off[n] if gw + 1 == GW else round_boundary(src_off, n, x1, decode)
    if pos >= end:
        return []
    s = warp_find_string(src_off, n, pos) if pos < src_off[n] else n
    tiles = []
    while pos < end and s < n:
        s0, s1 = src_off[s], src_off[s + 1]
        lim = s0 + (body_length(s1 - s0) if decode else s1 - s0)
        pos = max(pos, s0)
        if pos >= end:
            break
        if pos >= lim:
            s += 1
            continue
        b = min(pos + T, lim, end)
        tiles.append((s, pos, b))
        pos = b
    return tiles


def batch(seed, count, origin):
    g = np.random.default_rng(seed)
    lens = np.clip(np.rint(g.lognormal(np.log(200), 1.8, count)), 0, 60_000).astype(np.int64)
    lens[g.random(count) < 0.15] = 0
    lens[g.random(count) < 0.15] = g.integers(1, 7)
    off = np.concatenate([[0], np.cumsum(lens)]) + origin
    return [int(v) for v in off]


@pytest.mark.parametrize("decode", [False, True])
@pytest.mark.parametrize("seed,count,origin", [(1, 1, 0), (2, 5, 13), (3, 60, 0), (4, 300, 7),
                                               (5, 37, 1 << 20)])
def test_warps_cover_every_coded_byte_once(decode, seed, count, origin):
    src_off = batch(seed, count, origin)
    n = len(src_off) - 1
    g = 4 if decode else 3
    total = src_off[n] - src_off[0]
    unit = 16 if decode else 12                     # a tile is 32 lanes x U units
    for GW in sorted({1, 2, 3, 31, 32, 33, 608, 4864, max(1, total // 5)}):
        for T in (32 * 1 * unit, 32 * 8 * unit):
            covered = [[] for _ in range(n)]
            for gw in range(GW):
                for s, a, b in warp_tiles(src_off, n, gw, GW, T, decode):
                    s0, s1 = src_off[s], src_off[s + 1]
                    assert s0 <= a < b <= s1 and b - a <= T
                    assert (a - s0) % g == 0, (GW, gw, s, a)
                    covered[s].append((a, b))
            for s in range(n):
                s0, s1 = src_off[s], src_off[s + 1]
                lim = s0 + (body_length(s1 - s0) if decode else s1 - s0)
                spans = sorted(covered[s])
                at = s0
                for a, b in spans:
                    assert a == at, (GW, T, s, spans)
                    at = b
                assert at == lim, (GW, T, s, at, lim)


def test_search_finds_the_string_holding_each_byte():
    src_off = batch(9, 2000, 3)
    n = len(src_off) - 1
    g = np.random.default_rng(10)
    for x in list(g.integers(src_off[0], src_off[n], 3000)) + [src_off[0], src_off[n] - 1]:
        s = warp_find_string(src_off, n, int(x))
        assert s == bisect.bisect_right(src_off, int(x)) - 1
        assert src_off[s] <= x < src_off[s + 1]
