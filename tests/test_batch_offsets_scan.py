"""The three-launch exclusive scan of b64_batch_offsets, checked on the CPU.

1. Block b scans its 2048 capacities and writes their block-local exclusive
   offsets, except that its first slot gets the block's total.
2. One block of 1024 threads turns those totals into block prefixes in place,
   1024 totals a round with a running carry, and writes the grand total at n.
3. Block b adds its prefix (its first slot, now final) to its other slots.

Restated here with numpy at the block level and compared with a cumulative
sum, for string counts around the block size and past 1024 blocks (more than
two million strings, so that step 2 takes several rounds; the GPU tests use
up to 100,000 strings, one round).
"""
import numpy as np
import pytest

ITEMS, ROUND = 2048, 1024


def three_launch_scan(cap):
    n = cap.size
    dst = np.zeros(n + 1, np.int64)
    nblk = (n + ITEMS - 1) // ITEMS
    for b in range(nblk):                                   # 1. block-local
        first = b * ITEMS
        c = cap[first:min(first + ITEMS, n)]
        local = np.concatenate([[0], np.cumsum(c)[:-1]])
        local[0] = c.sum()
        dst[first:first + c.size] = local
    carry = 0                                               # 2. block totals, in rounds
    for base in range(0, nblk, ROUND):
        b = np.arange(base, base + ROUND)
        t = np.where(b < nblk, dst[np.minimum(b, max(nblk - 1, 0)) * ITEMS], 0) if nblk else \
            np.zeros(ROUND, np.int64)
        incl = np.cumsum(t)
        live = b < nblk
        dst[b[live] * ITEMS] = carry + incl[live] - t[live]
        carry += int(t.sum())
    dst[n] = carry
    for b in range(nblk):                                   # 3. fix-up
        first = b * ITEMS
        dst[first + 1:min(first + ITEMS, n)] += dst[first]
    return dst


@pytest.mark.parametrize("n", [0, 1, 2, 2047, 2048, 2049, 100_000, ITEMS * ROUND - 1,
                               ITEMS * ROUND, ITEMS * ROUND + 1, 2 * ITEMS * ROUND + 4097])
def test_matches_a_cumulative_sum(n):
    g = np.random.default_rng(n)
    cap = g.integers(0, 1 << 21, n).astype(np.int64)
    cap[g.random(n) < 0.1] = 0
    want = np.concatenate([[0], np.cumsum(cap)])
    assert np.array_equal(three_launch_scan(cap), want)
