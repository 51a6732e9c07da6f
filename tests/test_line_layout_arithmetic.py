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
segment's kSeg = 4096 raw bytes written as seg_q Q + seg_r. For L >= 16 a
lane decodes a unit of four whole groups (16 data characters) from three
8-byte loads at its raw offset rounded down to 8, taking each word either at
that offset or, past the one line break the unit can cross, e bytes further
on (that word shifted by e bytes into the next one, the next one past the 16
bytes being the low bytes of the last loaded word). A segment of a batched
document may sit delta bytes (0 to 15) past the staging buffer's start, where
its bulk copy put it: the unit path then reads it there (L >= 16, delta even
for CR LF) with delta added to the line start's offset. The data byte before
a segment is found by stepping back over the break from its start. These are
restated here with numpy and compared with the layout's definition over many
segments of every accepted layout. The GPU tests run the kernel itself on
L = 4, 64, 76 and 1020, and batched documents of several line lengths at
arbitrary starts.
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


def test_units_of_four_groups_take_their_characters_from_the_loaded_words():
    """For L >= 16: every unit of 16 data characters (its last groups inside
    the segment) is assembled from the 24 bytes loaded at its raw offset
    rounded down to 8, word by word from that offset or from e bytes further
    on (the words at or after the break, which falls between words), and the
    bytes are exactly the raw positions of its data characters. Each round of
    32 units writes its 12 output bytes a unit (at 12 i) below every load of
    the next round, and no load leaves the staging buffer."""
    for n, (L, e) in enumerate(le for le in LAYOUTS if le[0] >= 16):
        # a batched document's segment: delta bytes into the buffer, even for CR LF
        delta = n % 16 if e == 1 else 2 * (n % 8)
        Q = L + e
        inv = 0xFFFFFFFF // L + 1
        for s in range(0, 24 * K_SEG, K_SEG):
            k, r = divmod(s, Q)
            P = k * L + min(r, L)
            k1, r1 = divmod(s + K_SEG, Q)
            P1 = k1 * L + min(r1, L)
            rP = r if r < L else 0
            off0 = (-r if r < L else Q - r) + delta
            cA = (4 - P % 4) % 4
            nfull = (P1 - P - cA) // 4
            nunits = (nfull + 3) // 4
            i = np.arange(nunits, dtype=np.int64)
            ng = np.minimum(nfull - 4 * i, 4)
            t = rP + cA + 16 * i
            line = umulhi(t, inv).astype(np.int64)
            col = t - line * L
            assert np.all(col % 4 == 0)
            ro = off0 + line * e + t
            A, sh = ro & ~7, ro & 7
            assert np.all(sh + e <= 8)          # the shifted words' bytes stay in the 24 loaded
            assert np.all((sh & 3) + e <= 4)    # and the word past the 16 needs only its low word
            assert np.all(A >= 0) and np.all(A + 24 <= K_SEG + 48)  # inside the buffer
            tb = L - col
            b = np.arange(16, dtype=np.int64)
            got = ro[:, None] + b[None, :] + np.where(b[None, :] >= tb[:, None], e, 0)
            j = P + cA + 16 * i[:, None] + b[None, :]
            want = Q * (j // L) + j % L - s + delta
            used = b[None, :] < 4 * ng[:, None]
            assert np.array_equal(got[used], want[used]), (L, e, s, delta)
            assert np.all(want[used] < K_SEG + delta)  # whole groups inside the segment
            for r0 in range(0, nunits - 32, 32):
                wr_end = 12 * (r0 + 32)
                assert wr_end <= A[r0 + 32:r0 + 64].min(), (L, e, s, r0)


def test_data_byte_before_a_segment_by_stepping_back():
    """The data byte before a document's segment k > 0 (raw start S = 4096 k
    = line Q + column): one byte back, or 1 + e back where S starts a line,
    or column - L + 1 back where S lies inside the break. It is the raw
    position of data character P - 1, and no line division of P - 1 is
    needed."""
    for L, e in LAYOUTS:
        Q = L + e
        for k in range(1, 40):
            S = k * K_SEG
            line, col = divmod(S, Q)
            P = line * L + min(col, L)
            assert P > 0
            back = 1 + e if col == 0 else (col - L + 1 if col > L else 1)
            j = P - 1
            assert S - back == Q * (j // L) + j % L, (L, e, k)
