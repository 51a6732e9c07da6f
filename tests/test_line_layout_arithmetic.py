"""Index arithmetic of the line-layout fast path of the MIME decoder, checked
on the CPU for every layout the detector accepts (no GPU).

A document laid out as lines of L data characters (L a multiple of 4, 4 to
1020) each followed by a break of e bytes (CR LF: e = 2, LF: e = 1) has data
character j at raw position Q * (j div L) + j mod L, Q = L + e. The kernel
does not divide by L: it takes t div L as the high 32 bits of t * inv with
inv = floor((2^32 - 1) / L) + 1, valid for t < 2^13, and finds the raw offset
of data character P + d of a segment that starts at raw position S = k Q + r
as off0 + (t div L) e + t with t = rP + d (rP = r if r < L else 0; off0 = -r
if r < L else Q - r), and the segment's end as (k, r) advanced by the
segment's kSeg = 4096 raw bytes written as seg_q Q + seg_r. These are
restated here with numpy and compared with the layout's definition over many
segments of every accepted layout. The GPU tests run the kernel itself on
L = 4, 64, 76 and 1020.
"""
import numpy as np

K_SEG = 4096
LAYOUTS = [(L, e) for L in range(4, 1024, 4) for e in (1, 2)]


def umulhi(t, inv):
    return (t.astype(np.uint64) * np.uint64(inv)) >> np.uint64(32)


def test_reciprocal_division_is_exact_below_2_13():
    t = np.arange(1 << 13, dtype=np.uint64)
    for L in range(4, 1024, 4):
        inv = 0xFFFFFFFF // L + 1
        assert np.array_equal(umulhi(t, inv), t // np.uint64(L)), L


def test_raw_offsets_of_data_characters_in_every_segment():
    for L, e in LAYOUTS:
        Q = L + e
        inv = 0xFFFFFFFF // L + 1
        seg_q, seg_r = K_SEG // Q, K_SEG - (K_SEG // Q) * Q
        # the raw offsets all 4096 + L data characters after a segment start can need
        d = np.arange(K_SEG + L, dtype=np.int64)
        for s in range(0, 40 * K_SEG, K_SEG):
            k, r = divmod(s, Q)
            P = k * L + min(r, L)                      # data characters before the segment
            rP = r if r < L else 0
            off0 = -r if r < L else Q - r
            t = rP + d
            assert t.max() < (1 << 13)
            line = umulhi(t, inv).astype(np.int64)
            raw = off0 + line * e + t
            j = P + d
            want = Q * (j // L) + j % L - s
            assert np.array_equal(raw, want), (L, e, s)
            # the segment's end, advanced without a division
            k1, r1 = k + seg_q, r + seg_r
            if r1 >= Q:
                k1, r1 = k1 + 1, r1 - Q
            assert (k1, r1) == divmod(s + K_SEG, Q), (L, e, s)


def test_skipped_bytes_are_exactly_the_breaks():
    """The fast path checks raw offsets L - r + i Q (and the next byte for
    CR LF) as break bytes; they must be exactly the non-data positions of the
    segment."""
    for L, e in LAYOUTS:
        Q = L + e
        for s in range(0, 12 * K_SEG, K_SEG):
            r = s % Q
            rel = np.arange(L - r, K_SEG, Q)
            breaks = set()
            for x in rel:
                for b in range(e):
                    if 0 <= x + b < K_SEG:
                        breaks.add(int(x + b))
            pos = np.arange(s, s + K_SEG)
            data = (pos % Q) < L
            assert breaks == set((np.nonzero(~data)[0]).tolist()), (L, e, s)
