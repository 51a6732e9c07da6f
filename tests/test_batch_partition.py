"""How the batched kernels split and walk their work, checked on the CPU.

The concatenated input [src_off[0], src_off[n]) is cut into GW equal byte
ranges, one per warp. Each range end x is moved to the next 3-byte (encode)
or 4-character (decode) group boundary of the string holding x, found by a
32-way search over src_off in which every lane probes one of 32 evenly
spaced candidates and a ballot keeps the last that is <= x, but not past the
end of the string's coded part (encode: the whole string; decode: all but
its last 2..5 characters, which the finalize kernel decodes).

Within its range [P0, end) a warp cuts each string's part into units of G
bytes (12 encode, 16 decode; the last one shorter), numbers them in order
through a window of 32 strings (a warp scan of their unit counts), and walks
tiles of TB = 32 U G consecutive unit start positions. A tile's units are
coded in rounds: a whole tile of full units of one string at once; a round
whose strings' outputs are all aligned for a unit's stores (16 bytes encode,
4 decode) as consecutive units of whichever strings hold them (decode: 32 V
units, V a lane 32 apart, V = 4 with 8-unit tiles, else 2, when the tile
has that many left and every string of the window has aligned output;
otherwise up to 32, one a lane), each lane finding each
unit's string from the strings that start inside the round, stored straight
from registers; otherwise a string's units in the tile (a piece) in rounds
of their own, a string's shorter last unit by one lane after its full ones,
stored from registers when the string's output is aligned, else appended to
a pending run that is flushed when it breaks, fills or ends past a string's
last unit.
Warp ranges end on whole units. Packed and 16-byte aligned output offsets are
both run. The
kernel's rules are restated here in Python and run over batches with empty,
tiny and long strings, misaligned buffers and warp counts from 1 to more
warps than groups: every unit of every string must be coded exactly once,
with the right byte count, read from inside its tile's staging buffer and
stored inside the run buffer at an aligned offset, and every flushed run
must be exactly its units' outputs back to back. The GPU tests run the
kernels on the same kinds of batches.
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
    g = 16 if decode else 12                    # whole units
    r = (x - s0 + g - 1) // g * g
    return s0 + min(r, lim)


def shape(U, decode):
    G = 16 if decode else 12
    TB = 32 * U * G
    SIN = (TB + G + 48 + 15) & ~15
    return G, TB, SIN


class Window:
    """The kernel's window of 32 strings: per lane (string w0 + k) its
    segment start, first unit and unit count; the record's last-unit bytes."""

    def __init__(self, src_off, n, s, base, P0, end, decode, G):
        self.w0, self.base = s, base
        self.lo, self.us, self.un, self.nbl = [], [], [], []
        incl = 0
        for k in range(32):
            i = s + k
            valid = i < n
            lo = src_off[i] if valid else 0
            hi = src_off[i + 1] if valid else 0
            lim = lo + (body_length(hi - lo) if decode else hi - lo)
            sl, sh = max(lo, P0), min(lim, end)
            nb = sh - sl if valid and sh > sl else 0
            un = (nb + G - 1) // G
            self.lo.append(sl)
            self.us.append(base + incl)
            self.un.append(un)
            self.nbl.append(nb - (un - 1) * G if un else 0)
            incl += un
        self.end_u = base + incl
        self.next = src_off[min(s + 32, n)]

    def units_below(self, q, G):
        c = 0
        for k in range(32):
            dq = q - self.lo[k]
            if self.un[k] > 0 and dq > 0:
                c += min((dq + G - 1) // G, self.un[k])
        return self.base + c


def ballot_last(pred):
    mask = 0
    for k in range(32):
        if pred(k):
            mask |= 1 << k
    assert mask, "no window string holds the unit"
    return mask.bit_length() - 1


def out_bytes(nbu, G, padded, decode):
    """Output bytes of a unit of nbu input bytes (a short one is its string's last)."""
    if decode:
        return nbu // 4 * 3
    r = nbu % 3
    return nbu // 3 * 4 + (0 if r == 0 else 4 if padded else r + 1)


def warp_walk(src_off, n, gw, GW, U, decode, align, padded_of=lambda s: True, dst_off=None,
              mixed=True):
    V = (4 if U >= 8 else 2) if decode else 1   # units a lane in a wide mixed round
    """Yields (string, unit j, bytes, start, uniform) for every unit the warp
    codes, in order, and checks the tile, staging and output-run bounds on
    the way (the run's flushed spans are checked against the units' outputs)."""
    G, TB, SIN = shape(U, decode)
    O = 12 if decode else 16
    A = 4 if decode else 16          # alignment of a unit's store
    RUN = 32 * U * O
    origin, total = src_off[0], src_off[n] - src_off[0]
    if total <= 0:
        return
    x0 = origin + total * gw // GW
    x1 = origin + total * (gw + 1) // GW
    P0 = round_boundary(src_off, n, x0, decode)
    end = src_off[n] if gw + 1 == GW else round_boundary(src_off, n, x1, decode)
    if P0 >= end:
        return
    ntiles = (end - P0 + TB - 1) // TB
    win = Window(src_off, n, warp_find_string(src_off, n, P0), 0, P0, end, decode, G)
    g = 4 if decode else 3
    og = 3 if decode else 4
    run = {"dst": None, "len": 0, "units": []}   # pending run: start, bytes, units in it

    def seg_dst(k):
        s = win.w0 + k
        return dst_off[s] + (win.lo[k] - src_off[s]) // g * og

    def flush():
        # the run's bytes are exactly its units' outputs, back to back
        at = run["dst"]
        for (dst_at, nout) in run["units"]:
            assert dst_at == at
            at += nout
        assert at == run["dst"] + run["len"] and run["len"] <= RUN
        run.update(dst=None, len=0, units=[])

    R = 0
    for t in range(ntiles):
        p = P0 + t * TB
        q = min(p + TB, end)
        b = min(q + G - 1, end)
        pbase = p - ((align + p) & 15)
        span_end = ((align + b + 15) & ~15) - align      # staged bytes end (position)
        assert span_end - pbase <= SIN - 20, (span_end - pbase, SIN)
        while True:
            Rq = win.units_below(q, G)
            if Rq - R == 32 * U:       # the kernel's whole-tile path: one string, full units
                k0 = ballot_last(lambda k: win.un[k] > 0 and win.us[k] <= R)
                kq = ballot_last(lambda k: win.un[k] > 0 and win.us[k] <= Rq - 1)
                full0 = win.un[k0] - (1 if win.nbl[k0] < G else 0)
                if k0 == kq and Rq - win.us[k0] <= full0:
                    j0 = R - win.us[k0]
                    d0 = seg_dst(k0) + O * j0
                    direct = d0 % A == 0
                    if not direct:
                        if run["len"]:
                            flush()
                        run["dst"] = d0
                    for i in range(32 * U):
                        start = win.lo[k0] + G * (j0 + i)
                        o = start - pbase
                        assert p <= start < q and start + G <= b
                        assert 0 <= o and (o & ~15) + 32 <= SIN and o + 20 <= SIN
                        if direct:
                            assert (d0 + O * i) % A == 0
                        else:
                            run["units"].append((d0 + O * i, O))
                        yield win.w0 + k0, j0 + i, G, start, True
                    if not direct:
                        run["len"] = RUN
                    R = Rq
            while R < Rq:
                # wide only where every string of the window has aligned output
                wide = (V > 1 and Rq - R >= 32 * V and
                        all(win.un[k] == 0 or seg_dst(k) % A == 0 for k in range(32)))
                cnt = 32 * V if wide else min(32, Rq - R)
                has = [win.un[k] > 0 and win.us[k] < R + cnt and win.us[k] + win.un[k] > R
                       for k in range(32)]
                ok = mixed and all(win.un[k] == 0 or seg_dst(k) % A == 0
                                   for k in range(32) if has[k])
                NV = V if wide else 1
                if ok:
                    # a mixed round: lane l codes units R + 32 v + l (v < V) of
                    # whichever strings hold them, found from the strings
                    # starting inside the round (V block masks and a slot array)
                    ks0 = ballot_last(lambda kk: win.un[kk] > 0 and win.us[kk] <= R)
                    slot, B = {}, [0] * NV
                    for k in range(32):
                        if has[k] and win.us[k] > R:
                            d = win.us[k] - R
                            assert d < 32 * NV
                            slot[d] = k
                            B[d >> 5] |= 1 << (d & 31)
                    carry = ks0
                    for v in range(NV):
                        for lane in range(32):
                            i = 32 * v + lane
                            m = B[v] & ((2 << lane) - 1)
                            k = slot[32 * v + m.bit_length() - 1] if m else carry
                            if i >= cnt:
                                continue        # idle: reads the buffer's start, stores nothing
                            assert win.us[k] <= R + i < win.us[k] + win.un[k]
                            j = R + i - win.us[k]
                            part = j + 1 == win.un[k] and win.nbl[k] < G
                            nbu = win.nbl[k] if part else G
                            start = win.lo[k] + G * j
                            assert p <= start < q and start + nbu <= b, (p, q, start, nbu, b)
                            o = start - pbase
                            assert 0 <= o and (o & ~7) + 24 <= SIN and o + 20 <= SIN
                            assert (seg_dst(k) + O * j) % A == 0
                            yield win.w0 + k, j, nbu, start, not part
                        if B[v]:
                            carry = slot[32 * v + B[v].bit_length() - 1]
                    R += cnt
                    continue
                k = ballot_last(lambda kk: win.un[kk] > 0 and win.us[kk] <= R)
                us, un, nbl = win.us[k], win.un[k], win.nbl[k]
                pend = min(Rq, us + un)
                padded = padded_of(win.w0 + k)
                direct = seg_dst(k) % A == 0
                out_last = out_bytes(nbl, G, padded, decode) if nbl < G else O

                def run_at(d, need):
                    if run["len"] and (run["dst"] + run["len"] != d or run["len"] % A or
                                       run["len"] + need > RUN):
                        flush()
                    if run["len"] == 0:
                        run["dst"] = d

                while R < pend:                 # 32 units a round, one string
                    cnt = min(32, pend - R)
                    j0 = R - us
                    ends = R + cnt == us + un and nbl < G
                    if not direct:
                        run_at(seg_dst(k) + O * j0, 32 * O)
                    for lane in range(cnt):
                        j = j0 + lane
                        part = ends and lane + 1 == cnt
                        nbu = nbl if part else G
                        assert part or j + 1 < un or nbl == G
                        start = win.lo[k] + G * j
                        assert p <= start < q and start + nbu <= b, (p, q, start, nbu, b)
                        o = start - pbase
                        assert 0 <= o and o + 20 <= SIN and (o & ~15) + 32 <= SIN
                        nout = out_last if part else O
                        if direct:
                            assert (seg_dst(k) + O * j) % A == 0
                        else:
                            so = run["len"] + O * lane     # the lane's store in the run buffer
                            assert so % A == 0 and so + O <= RUN
                            run["units"].append((seg_dst(k) + O * j, nout))
                        yield win.w0 + k, j, nbu, start, not part
                    if not direct:
                        run["len"] += O * (cnt - 1) + out_last if ends else O * cnt
                    R += cnt
            if Rq < win.end_u or win.w0 + 32 >= n or win.next >= q:
                break
            win = Window(src_off, n, win.w0 + 32, win.end_u, P0, end, decode, G)
    if run["len"]:
        flush()


def batch(seed, count, origin):
    g = np.random.default_rng(seed)
    lens = np.clip(np.rint(g.lognormal(np.log(200), 1.8, count)), 0, 60_000).astype(np.int64)
    lens[g.random(count) < 0.15] = 0
    lens[g.random(count) < 0.15] = g.integers(1, 7)
    off = np.concatenate([[0], np.cumsum(lens)]) + origin
    return [int(v) for v in off]


@pytest.mark.parametrize("decode", [False, True])
@pytest.mark.parametrize("seed,count,origin", [(1, 1, 0), (2, 5, 13), (3, 60, 0), (4, 300, 7),
                                               (5, 37, 1 << 20), (6, 900, 3)])
def test_warps_code_every_unit_once(decode, seed, count, origin):
    src_off = batch(seed, count, origin)
    n = len(src_off) - 1
    G = 16 if decode else 12
    g = 4 if decode else 3
    total = src_off[n] - src_off[0]
    lens = [src_off[i + 1] - src_off[i] for i in range(n)]
    padded = [i % 3 != 1 for i in range(n)]
    if decode:
        caps = [(m + 3) // 4 * 3 for m in lens]
    else:
        caps = [(m + 2) // 3 * 4 if padded[i] else (4 * m + 2) // 3 for i, m in enumerate(lens)]
    layouts = []
    for align16 in (False, True):   # packed outputs, and 16-byte aligned string starts
        dst_off = [0]
        for c in caps:
            dst_off.append(dst_off[-1] + ((c + 15) // 16 * 16 if align16 else c))
        layouts.append(dst_off)
    for GW, dst_off in [(gw, layouts[i % 2]) for i, gw in
                        enumerate(sorted({1, 2, 3, 31, 33, 608, max(1, total // 5)}))]:
        for U, align, mixed in ((1, 0, True), (4, 5, False), (8, 12, True), (8, 3, False)):
            seen = [dict() for _ in range(n)]     # string -> {byte offset: bytes}
            uniform_rounds = 0
            for gw in range(GW):
                for s, j, nbu, start, uniform in warp_walk(src_off, n, gw, GW, U, decode, align,
                                                           lambda i: padded[i], dst_off, mixed):
                    rel = start - src_off[s]
                    assert rel % g == 0
                    assert rel not in seen[s], (GW, U, s, rel)
                    seen[s][rel] = nbu
                    uniform_rounds += uniform
            for s in range(n):
                ln = src_off[s + 1] - src_off[s]
                lim = body_length(ln) if decode else ln
                at = 0
                for rel in sorted(seen[s]):
                    assert rel == at, (GW, U, s, rel, at)
                    at += seen[s][rel]
                    # whole groups except at the string's end (encode)
                    assert seen[s][rel] % g == 0 or at == ln, (s, rel, seen[s][rel])
                assert at == lim, (GW, U, s, at, lim)
            if GW <= 3 and total > 100_000:
                assert uniform_rounds > 0


def test_search_finds_the_string_holding_each_byte():
    src_off = batch(9, 2000, 3)
    n = len(src_off) - 1
    g = np.random.default_rng(10)
    for x in list(g.integers(src_off[0], src_off[n], 3000)) + [src_off[0], src_off[n] - 1]:
        s = warp_find_string(src_off, n, int(x))
        assert s == bisect.bisect_right(src_off, int(x)) - 1
        assert src_off[s] <= x < src_off[s + 1]
