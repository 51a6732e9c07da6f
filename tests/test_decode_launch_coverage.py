"""Launch shapes of the single-buffer decode, checked on the CPU: every group
of four characters before the tail is decoded by exactly one thread.

Inputs up to 512 KiB: one 1024-thread block up to 32 KiB, else a cluster of
ceil(m / 8 KiB) blocks capped at the device's cluster limit (8, or up to 16
where the non-portable size is co-scheduled) and raised to 2; thread g of
the cluster takes groups g, g + stride, ... (at most 16). Larger inputs: a
persistent grid in which warp gw takes chunks gw, gw + GW, ... and warp
n_chunks mod GW the groups after the last whole chunk. Restated here from
the launch rules; the GPU tests run the kernels at these sizes.
"""
import pytest

K_SMALL_THREADS, K_SMALL_PER = 1024, 16
K_SMALL_MAX, K_SMALL_SINGLE, K_SMALL_CTA_BYTES = 512 << 10, 32 << 10, 8 << 10


def body_length(m):
    return (m - 2) & ~3 if m >= 2 else 0


def small_ctas(m, limit):
    want = min((m + K_SMALL_CTA_BYTES - 1) // K_SMALL_CTA_BYTES, limit)
    return 1 if m <= K_SMALL_SINGLE else max(want, 2)


@pytest.mark.parametrize("limit", [8, 9, 12, 16])
def test_small_launch_holds_every_group(limit):
    sizes = set(range(0, 70_000, 997)) | {K_SMALL_SINGLE + d for d in (-5, -1, 0, 1, 2, 5)}
    sizes |= {K_SMALL_MAX + d for d in (-6, -2, -1, 0)} | {141_020, 247_222, 2_357, 3_144}
    for m in sorted(sizes):
        if m > K_SMALL_MAX:
            continue
        ctas = small_ctas(m, limit)
        assert 1 <= ctas <= max(limit, 2)
        stride = ctas * K_SMALL_THREADS
        quads = body_length(m) // 4
        assert quads <= K_SMALL_PER * stride, (m, ctas)     # every group has a thread


@pytest.mark.parametrize("chunk", [1024, 2048])
def test_body_chunks_and_leftover_are_taken_once(chunk):
    warps = 16
    for body in (0, 4, chunk - 4, chunk, chunk + 4, 7 * chunk + 12, 1000 * chunk + 4 * 37):
        n_chunks = body // chunk
        for ctas in (1, 2, 3, 152, 304):
            grid = min(ctas, max(1, (n_chunks + warps - 1) // warps))
            GW = grid * warps
            taken = []
            for gw in range(GW):
                K = (n_chunks - 1 - gw) // GW + 1 if gw < n_chunks else 0
                taken += [gw + k * GW for k in range(K)]
            assert sorted(taken) == list(range(n_chunks)), (body, ctas)
            leftover_warps = [gw for gw in range(GW) if gw == n_chunks % GW]
            assert len(leftover_warps) == 1                 # the groups after the chunks
