"""Segment slots of the batched MIME decoder, checked on the CPU.

Document d's ceil(len_d / 4096) segments keep their state words at slots
doc_slot(d) + k with doc_slot(d) = (src_off[d] - src_off[0]) div 4096 + d,
and the workspace holds (src_off[n] - src_off[0]) div 4096 + n + 1 slots.
Each warp walks its own equal, contiguous range of slots, skipping slots no
document uses and finding a slot's document by a search that it repeats only
when the walk leaves the remembered document. Restated here in Python and
run over batches with empty, tiny and multi-segment documents: the slot
ranges of the documents never overlap and fit the workspace, the walks of
all warps visit every (document, segment) exactly once, and the one-pass and
counting passes, each walking only its own documents, split them between
them.
"""
import bisect

import numpy as np
import pytest

K_SEG = 4096


def doc_slot(src_off, d):
    return (src_off[d] - src_off[0]) // K_SEG + d


def doc_slots(src_off, n):
    return (src_off[n] - src_off[0]) // K_SEG + n + 1


def nseg(src_off, d):
    return (src_off[d + 1] - src_off[d] + K_SEG - 1) // K_SEG


def find_doc(src_off, n, g):
    """The largest d in [0, n) with doc_slot(d) <= g."""
    slots = [doc_slot(src_off, d) for d in range(n)]
    return bisect.bisect_right(slots, g) - 1


def walk(src_off, n, warp, warps, counted_of=None, counted=False):
    """counted_of: a pass's filter (the kernel's kDocCounted bit per
    document); only the documents whose bit equals `counted` are walked."""
    nslots = doc_slots(src_off, n)
    per = (nslots + warps - 1) // warps
    g = min(warp * per, nslots)
    g1 = min(g + per, nslots)
    d, first, ns = -1, 0, 0
    out = []
    while g < g1:
        if d < 0 or g < first or g >= first + ns:
            if d >= 0 and g >= first + ns and d + 1 < n and g < doc_slot(src_off, d + 1):
                g += 1
                continue
            d = find_doc(src_off, n, g)
            first, ns = doc_slot(src_off, d), nseg(src_off, d)
            if counted_of is not None and counted_of[d] != counted:
                ns = 0                  # not this pass's document: skip its slots
            if g >= first + ns:
                g += 1
                continue
        out.append((d, g - first, g))
        g += 1
    return out


def batch(seed, count, origin):
    g = np.random.default_rng(seed)
    lens = np.rint(g.lognormal(np.log(3000), 1.6, count)).astype(np.int64)
    lens = np.clip(lens, 0, 200_000)
    lens[g.random(count) < 0.2] = 0
    lens[g.random(count) < 0.2] = g.integers(1, 40)
    lens[g.random(count) < 0.1] = K_SEG * g.integers(1, 4)      # exact multiples
    off = np.concatenate([[0], np.cumsum(lens)]) + origin
    return [int(v) for v in off]


@pytest.mark.parametrize("seed,count,origin", [(1, 1, 0), (2, 7, 5), (3, 200, 0),
                                               (4, 64, 4095), (5, 300, 1 << 20)])
def test_slot_ranges_are_disjoint_and_fit_the_workspace(seed, count, origin):
    src_off = batch(seed, count, origin)
    n = len(src_off) - 1
    cap = doc_slots(src_off, n)
    end = -1
    for d in range(n):
        first = doc_slot(src_off, d)
        assert first > end or nseg(src_off, d) == 0, d
        if nseg(src_off, d):
            end = first + nseg(src_off, d) - 1
    assert end < cap
    # the library's workspace size: 3 status words a document, one word that
    # says whether any document needs the counting passes, a state and a
    # layout word a document, then the slots
    from paper_1910_05109_gb300 import binding, build
    build.build()
    total = src_off[n] - src_off[0]
    assert binding.lib().b64_mime_batch_workspace_size(n, total) == 8 * (5 * n + 1 + cap)


@pytest.mark.parametrize("seed,count,origin", [(1, 1, 0), (2, 7, 5), (3, 200, 0),
                                               (4, 64, 4095), (5, 300, 1 << 20)])
def test_warp_walks_visit_every_segment_once(seed, count, origin):
    src_off = batch(seed, count, origin)
    n = len(src_off) - 1
    want = {(d, k) for d in range(n) for k in range(nseg(src_off, d))}
    for warps in sorted({1, 2, 5, 32, 1216, doc_slots(src_off, n) + 3}):
        seen = []
        for w in range(warps):
            for d, k, g in walk(src_off, n, w, warps):
                assert g == doc_slot(src_off, d) + k
                seen.append((d, k))
        assert len(seen) == len(set(seen)) and set(seen) == want, warps


@pytest.mark.parametrize("seed,count,origin", [(2, 7, 5), (3, 200, 0), (5, 300, 1 << 20)])
def test_the_two_passes_split_the_documents(seed, count, origin):
    """The one-pass walk (documents with a line layout) and the counting
    passes' walk (the others) together visit every segment exactly once, and
    each only its own documents' segments."""
    src_off = batch(seed, count, origin)
    n = len(src_off) - 1
    counted_of = [bool(b) for b in np.random.default_rng(seed + 9).random(n) < 0.3]
    want = {(d, k) for d in range(n) for k in range(nseg(src_off, d))}
    for warps in (1, 5, 32, 1216):
        seen = []
        for counted in (False, True):
            for w in range(warps):
                for d, k, g in walk(src_off, n, w, warps, counted_of, counted):
                    assert counted_of[d] == counted and g == doc_slot(src_off, d) + k
                    seen.append((d, k))
        assert len(seen) == len(set(seen)) and set(seen) == want, warps
