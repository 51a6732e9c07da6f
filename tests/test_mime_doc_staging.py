"""Staging of a batched MIME document's segment, checked on the CPU.

A segment's 16-byte aligned span lands at buf + kLead by one bulk copy, so
segment byte i sits at buf[kLead + pd + i] (pd = the segment's address mod
16). Where the line path cannot read it there, the warp moves it down in
place, a row at a time: in row r, lane l reads the 16 bytes at pd + 512 r +
16 l (two aligned 16-byte words and a funnel shift; bytes at or past the
segment's length read as spaces), all lanes read before any writes, then
lane l writes them at 512 r + 16 l. Here the 32 lanes are simulated read by
read and write by write: the result is the segment at buf + kLead, and no
write lands on a byte that a later read of the same move still needs. Also
which segments the line path reads in place: whole segments with lines of
at least 16 characters and, with CR LF breaks, an even pd.
"""
import numpy as np

K_LEAD, K_ROW, K_ROWS = 16, 512, 8
K_SEG = K_ROW * K_ROWS
K_BUF = K_LEAD + K_SEG + 48


def move_down(buf: np.ndarray, pd: int, length: int):
    """The in-place move; returns the buffer and the byte positions each
    read took from and each write went to, in program order."""
    raw = K_LEAD
    events = []                                   # (kind, row, lane, positions)
    for r in range(K_ROWS):
        vals = []
        for lane in range(32):                    # every lane's reads of row r
            off = K_ROW * r + 16 * lane
            if off + 16 <= length:
                a = raw + ((pd + off) & ~15)      # the two aligned words it loads
                pos = list(range(a, a + (32 if (pd + off) & 15 else 16)))
                v = buf[raw + pd + off: raw + pd + off + 16].copy()
            else:
                pos = [raw + pd + off + j for j in range(16) if off + j < length]
                v = np.array([buf[raw + pd + off + j] if off + j < length else 0x20
                              for j in range(16)], np.uint8)
            events.append(("r", r, lane, pos))
            vals.append(v)
        for lane in range(32):                    # then its writes (after __syncwarp)
            off = K_ROW * r + 16 * lane
            buf[raw + off: raw + off + 16] = vals[lane]
            events.append(("w", r, lane, list(range(raw + off, raw + off + 16))))
    return buf, events


def test_move_down_gives_the_segment_and_never_clobbers_a_pending_read():
    g = np.random.default_rng(5)
    for pd in range(16):
        for length in (K_SEG, K_SEG - 1, 3000, 17, 1):
            seg = g.integers(0, 256, length, dtype=np.uint8)
            buf = g.integers(0, 256, K_BUF, dtype=np.uint8)
            span = np.frombuffer(bytes(buf[K_LEAD:K_LEAD + pd]) + seg.tobytes(), np.uint8)
            buf[K_LEAD:K_LEAD + span.size] = span
            assert K_LEAD + pd + K_SEG + 16 <= K_BUF       # every load inside the buffer
            out, events = move_down(buf.copy(), pd, length)
            want = np.concatenate([seg, np.full(K_SEG - length, 0x20, np.uint8)])
            assert np.array_equal(out[K_LEAD:K_LEAD + K_SEG], want), (pd, length)
            # a write may not reach a byte that a read after it (in program
            # order across the warp's rows) takes
            written = set()
            for kind, r, lane, pos in events:
                if kind == "w":
                    written.update(pos)
                else:
                    assert not written.intersection(
                        p for p in pos if p < K_LEAD + pd + length), (pd, length, r, lane)


def line_path_reads_in_place(seg_len: int, L: int, eol: int, pd: int) -> bool:
    return seg_len == K_SEG and L >= 16 and (eol == 1 or pd % 2 == 0)


def test_which_segments_are_read_in_place():
    assert line_path_reads_in_place(K_SEG, 76, 2, 6)
    assert not line_path_reads_in_place(K_SEG, 76, 2, 7)    # CR LF, odd offset: moved
    assert line_path_reads_in_place(K_SEG, 64, 1, 7)        # LF: any offset
    assert not line_path_reads_in_place(K_SEG, 12, 1, 0)    # short lines: one group a lane
    assert not line_path_reads_in_place(K_SEG - 1, 76, 2, 0)  # a document's last segment
