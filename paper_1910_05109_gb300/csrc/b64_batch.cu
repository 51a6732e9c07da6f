// Batched variable-length encode and strict decode: many independent strings
// in one persistent launch (the paper's codec, Sec. 3.1 and Sec. 3.2, applied
// per string; batching itself is not in the paper).
//
// String i is src[src_off[i] .. src_off[i+1]) and goes to dst + dst_off[i],
// with its own alphabet (one of up to kMaxAlphabets passed by value). Work is
// cut into tiles of one warp each: 32 x U units of 12 input bytes (encode) or
// 16 characters (decode), U chosen at launch (the autotuner's tile size).
//
// Launch sequence (all on one stream, so it can be recorded in a CUDA graph):
//   1. encode: one thread per string writes the string's output length to
//      results; decode: the per-string error words in the caller's workspace
//      are set to "none" (a memset);
//   2. tile kernel (persistent): the concatenated input is split into equal
//      byte ranges, one per warp. A warp finds the strings that hold its
//      range ends with a 32-way search over src_off and moves both ends up to
//      the next 3-byte (encode) or 4-character (decode) group boundary of
//      their string, so neighbouring warps meet without talking to each other
//      and no per-string scan is needed. It then walks its range string by
//      string in tiles of at most 32 x U units. A tile is brought into the
//      warp's shared memory by a bulk (TMA) copy of its 16-byte aligned span
//      (the next tile's copy is started before the current one is coded), or
//      staged with aligned loads where the span would leave the source
//      buffer, re-aligned with funnel shifts, coded with the same per-unit
//      steps as the single-buffer kernels, and copied out with aligned 16-byte
//      stores and byte stores at the edges. Decode tiles fold bad-byte offsets
//      into the string's error word with an atomic minimum;
//   3. decode only: one thread per string applies the padding and length
//      rules to the string's last 2..5 characters and writes its result.
#include <mutex>

#include "b64_internal.h"
#include "b64_smem.cuh"

namespace b64 {
namespace {


#ifndef B64_BATCH_STAGES
#define B64_BATCH_STAGES 2
#endif

// The tile kernels' shape for U units a lane: 8 warps a block (4 for U = 8,
// measured faster there), each with a ring of kStages input staging buffers
// (kStages - 1 tiles in flight while one is coded) and one output buffer, in
// dynamic shared memory. Two stages: three and four measured no faster (the
// kernels are bound by instruction issue, not by the latency of the copies)
// and cost resident blocks. The encoder keeps the 64-entry table: the
// character-pair table of the single-buffer encoder measured slower here
// (its 8 KiB a block cost resident blocks).
template <int U, bool kDecode>
struct TileShape {
    static constexpr int kWarps = U >= 8 ? 4 : 8;
    static constexpr int kThreads = 32 * kWarps;
    static constexpr int kStages = B64_BATCH_STAGES;
    static constexpr uint32_t T = kDecode ? 32 * U * 16 : 32 * U * 12;  // input per tile
    static constexpr uint32_t TO = kDecode ? T / 4 * 3 : T / 3 * 4 + 4;  // output (+ padding)
    static constexpr uint32_t SIN = T + 32;                    // room for a ragged start
    static constexpr uint32_t SOUT = (TO + 16 + 15) & ~15u;     // rows stay 16-byte aligned
    static constexpr size_t kSmem = size_t(kWarps) * (size_t(kStages) * SIN + SOUT);
    static_assert(SIN % 16 == 0 && kStages >= 2 && kStages <= 32, "staging ring");
};

__host__ __device__ __forceinline__ uint64_t dec_body_length(uint64_t m) {
    return m >= 2 ? ((m - 2) & ~uint64_t(3)) : 0;
}

__host__ __device__ __forceinline__ uint64_t enc_length(uint64_t n, int padded) {
    const uint64_t g = n / 3, r = n % 3;
    return r == 0 ? 4 * g : 4 * g + (padded ? 4 : r + 1);
}

// ------------------------------------------------------------------ staging helpers
// Copies bytes [a, b) of global memory into sbuf so that byte a lands at
// sbuf[a & 15]; every 16-byte piece that lies inside [lo, hi) (the whole
// source buffer) is moved with one aligned 16-byte load, the ragged pieces at
// the buffer's own edges byte by byte. Warp-collective.
__device__ __forceinline__ void warp_stage_in(uint8_t* sbuf, const uint8_t* base, uint64_t a,
                                              uint64_t b, uint64_t lo_b, uint64_t hi_b, int lane) {
    const uintptr_t pa = reinterpret_cast<uintptr_t>(base + a) & ~uintptr_t(15);
    const uintptr_t pb = (reinterpret_cast<uintptr_t>(base + b) + 15) & ~uintptr_t(15);
    const uintptr_t lo = reinterpret_cast<uintptr_t>(base + lo_b);
    const uintptr_t hi = reinterpret_cast<uintptr_t>(base + hi_b);
    const int pieces = int((pb - pa) >> 4);
    for (int k = lane; k < pieces; k += 32) {
        const uintptr_t p = pa + 16 * uintptr_t(k);
        if (p >= lo && p + 16 <= hi) {
            *reinterpret_cast<uint4*>(sbuf + 16 * k) = *reinterpret_cast<const uint4*>(p);
        } else {
            for (int i = 0; i < 16; ++i)
                if (p + i >= lo && p + i < hi)
                    sbuf[16 * k + i] = *reinterpret_cast<const uint8_t*>(p + i);
        }
    }
}

__device__ uint32_t g_fault;

// Lane 0 only: if the 16-byte aligned span around [a, b) lies inside the
// source buffer [0, src_end), start one bulk (TMA) copy of it into sbuf
// (byte a lands at sbuf[(base + a) & 15], as warp_stage_in places it),
// completing on `bar`, and return true; otherwise return false and the warp
// stages the tile itself when it gets to it.
__device__ __forceinline__ bool issue_tile_load(uint8_t* sbuf, const uint8_t* base, uint64_t a,
                                                uint64_t b, uint64_t src_end, uint64_t* bar) {
    const uintptr_t pa = reinterpret_cast<uintptr_t>(base + a) & ~uintptr_t(15);
    const uintptr_t pb = (reinterpret_cast<uintptr_t>(base + b) + 15) & ~uintptr_t(15);
    if (pa < reinterpret_cast<uintptr_t>(base) ||
        pb > reinterpret_cast<uintptr_t>(base + src_end) || pb == pa)
        return false;
    const uint32_t bytes = uint32_t(pb - pa);
    mbar_arrive_expect_tx(bar, bytes);
    bulk_load(sbuf, reinterpret_cast<const void*>(pa), bytes, bar);
    return true;
}

// Makes tile t's staged bytes available in sbuf: waits for its bulk copy
// (bounded), or stages it now. Returns false if the wait ran out.
__device__ __forceinline__ bool tile_ready(bool by_copy, uint8_t* sbuf, uint64_t* bar,
                                           uint32_t& phases, int k, const uint8_t* base,
                                           uint64_t a, uint64_t b, uint64_t src_end, int lane) {
    if (by_copy) {
        const bool ok = mbar_wait(bar, (phases >> k) & 1u);
        phases ^= 1u << k;
        return __all_sync(0xffffffffu, ok);
    }
    warp_stage_in(sbuf, base, a, b, 0, src_end, lane);
    fence_proxy_async_smem();  // before a later bulk copy reuses this buffer
    __syncwarp();
    return true;
}

// Writes sbuf[0 .. len) to global q (any alignment): aligned 16-byte stores
// for the middle, byte stores for the ragged head and tail. Warp-collective.
__device__ __forceinline__ void warp_stage_out(uint8_t* q, const uint8_t* sbuf, uint32_t len,
                                               int lane) {
    const uint32_t head = uint32_t((16 - (reinterpret_cast<uintptr_t>(q) & 15)) & 15);
    const uint32_t h = head < len ? head : len;
    if (lane < int(h)) q[lane] = sbuf[lane];
    const uint32_t body = (len - h) & ~15u;
    for (uint32_t k = lane; k < body / 16; k += 32) {
        const uint32_t off = h + 16 * k;
        *reinterpret_cast<uint4*>(q + off) = load16_shifted_u(sbuf, off);
    }
    for (uint32_t i = h + body + lane; i < len; i += 32) q[i] = sbuf[i];
}

// Warp-cooperative search: the largest string s in [0, n) with
// src_off[s] <= x, for src_off[0] <= x < src_off[n] (that string is never
// empty). Each round every lane probes one of 32 evenly spaced candidates.
__device__ __forceinline__ int64_t warp_find_string(const int64_t* __restrict__ src_off,
                                                    int64_t n, int64_t x, int lane) {
    int64_t lo = 0, hi = n;  // src_off[lo] <= x < src_off[hi]
    while (hi - lo > 1) {
        const int64_t step = (hi - lo + 31) / 32;
        const int64_t probe = lo + int64_t(lane) * step;
        const bool le = probe < hi && src_off[probe] <= x;
        const uint32_t mask = __ballot_sync(0xffffffffu, le);
        const int k = 31 - __clz(mask);  // lane 0 always holds (probe = lo)
        const int64_t nlo = lo + int64_t(k) * step;
        const int64_t nhi = nlo + step < hi ? nlo + step : hi;
        lo = nlo;
        hi = nhi;
    }
    return lo;
}

// Where a warp's range boundary at byte x (src_off coordinates) really falls:
// rounded up to the next group boundary (3 bytes for encode, 4 characters for
// decode) of the string that holds x, but not past the end of the string's
// coded part (its end; for decode, its body). Every warp rounds the same way,
// so neighbouring ranges meet exactly.
template <bool kDecode>
__device__ __forceinline__ int64_t round_boundary(const int64_t* __restrict__ src_off, int64_t n,
                                                  int64_t x, int lane) {
    if (x >= src_off[n]) return src_off[n];
    const int64_t s = warp_find_string(src_off, n, x, lane);
    const int64_t s0 = src_off[s];
    const int64_t len = src_off[s + 1] - s0;
    const int64_t lim = kDecode ? int64_t(dec_body_length(uint64_t(len))) : len;
    constexpr int64_t g = kDecode ? 4 : 3;
    const int64_t r = (x - s0 + g - 1) / g * g;
    return s0 + (r < lim ? r : lim);
}

// The per-string metadata of strings [w0, w0 + 32), one string per lane
// (loaded with one coalesced round, read back by shuffles).
struct Window {
    int64_t w0 = INT64_MIN / 2;     // no string loaded yet
    int64_t lo = 0, hi = 0, d = 0;  // src_off[i], src_off[i + 1], dst_off[i]
    uint32_t id = 0;                // alphabet of string i
    __device__ __forceinline__ void load(int64_t s, const int64_t* __restrict__ src_off,
                                         const int64_t* __restrict__ dst_off,
                                         const uint8_t* __restrict__ alph_id, int64_t n,
                                         int lane) {
        w0 = s;
        const int64_t i = s + lane;
        lo = i < n ? src_off[i] : 0;
        hi = i < n ? src_off[i + 1] : 0;
        d = i < n ? dst_off[i] : 0;
        id = (i < n && alph_id) ? uint32_t(alph_id[i] & (kMaxAlphabets - 1)) : 0u;
    }
};

// One tile: bytes [a, b) of string s, with the string's metadata.
struct Tile {
    int64_t s = 0, a = 0, b = 0, s0 = 0, s1 = 0, d0 = 0;
    uint32_t id = 0;
};

// The warp's walk over its range [pos, end): strings in order, tiles of at
// most T bytes, each starting on a group boundary of its string.
// Warp-collective (every lane holds the same state).
template <bool kDecode>
struct Cursor {
    int64_t s, pos, end;
    Window win;
    __device__ __forceinline__ bool next(const int64_t* __restrict__ src_off,
                                         const int64_t* __restrict__ dst_off,
                                         const uint8_t* __restrict__ alph_id, int64_t n, int64_t T,
                                         int lane, Tile* t) {
        for (;;) {
            if (pos >= end || s >= n) return false;
            if (s < win.w0 || s >= win.w0 + 32) win.load(s, src_off, dst_off, alph_id, n, lane);
            const int k = int(s - win.w0);
            const int64_t s0 = __shfl_sync(0xffffffffu, win.lo, k);
            const int64_t s1 = __shfl_sync(0xffffffffu, win.hi, k);
            const int64_t len = s1 - s0;
            const int64_t lim = s0 + (kDecode ? int64_t(dec_body_length(uint64_t(len))) : len);
            if (pos < s0) pos = s0;
            if (pos >= end) return false;
            if (pos >= lim) {  // string done (or empty): on to the next one
                ++s;
                continue;
            }
            int64_t b = pos + T;
            if (b > lim) b = lim;
            if (b > end) b = end;
            t->s = s;
            t->a = pos;
            t->b = b;
            t->s0 = s0;
            t->s1 = s1;
            t->d0 = __shfl_sync(0xffffffffu, win.d, k);
            t->id = __shfl_sync(0xffffffffu, win.id, k);
            pos = b;
            return true;
        }
    }
};

// The warp's walk over its tiles with a ring of S staging buffers: the next
// S - 1 tiles are described (by the warp-uniform cursor) and their bulk
// copies started before the current one is coded; lane 0 keeps each tile's
// description in the warp's ring in shared memory. process(t, sin) codes
// one staged tile. Returns false if a bulk copy did not arrive in time.
template <bool kDecode, int S, class Process>
__device__ __forceinline__ bool walk_tiles(Cursor<kDecode>& cur, const uint8_t* __restrict__ src,
                                           const int64_t* __restrict__ src_off,
                                           const int64_t* __restrict__ dst_off,
                                           const uint8_t* __restrict__ alph_id, int64_t n,
                                           int64_t T, uint64_t src_end, uint8_t* sin_base,
                                           uint32_t sin_stride, uint64_t* bars, Tile* ring,
                                           uint32_t* ring_copy, int lane, Process process) {
    bool more = true;
    int64_t issued = 0;
    auto issue = [&](int slot) {
        Tile nt;
        if (!cur.next(src_off, dst_off, alph_id, n, T, lane, &nt)) return false;
        if (lane == 0) {
            ring_copy[slot] = issue_tile_load(sin_base + size_t(slot) * sin_stride, src,
                                              uint64_t(nt.a), uint64_t(nt.b), src_end, &bars[slot]);
            ring[slot] = nt;
        }
        return true;
    };
    for (int k = 0; k < S - 1 && more; ++k) {
        more = issue(k);
        issued += more;
    }
    uint32_t phases = 0;
    for (int64_t it = 0; it < issued; ++it) {
        const int k = int(it % S);
        fence_proxy_async_smem();  // this lane's reads of tile it - 1 before the copy below
        __syncwarp();              // every lane is done with tile it - 1's buffer and ring slot
        if (more) {
            more = issue(int((it + S - 1) % S));
            issued += more;
        }
        __syncwarp();              // ring writes of lane 0 are visible
        const Tile t = ring[k];
        const bool by_copy = ring_copy[k] != 0;
        uint8_t* sin = sin_base + size_t(k) * sin_stride;
        if (!tile_ready(by_copy, sin, &bars[k], phases, k, src, uint64_t(t.a), uint64_t(t.b),
                        src_end, lane)) {
            // let this copy and the later ones in flight land (bounded) before
            // the block can exit; this tile's wait already flipped its parity
            if (lane == 0)
                for (int64_t i = it; i < issued; ++i) {
                    const int kk = int(i % S);
                    if (ring_copy[kk])
                        mbar_wait(&bars[kk], ((phases >> kk) & 1u) ^ (i == it ? 1u : 0u));
                }
            return false;
        }
        process(t, sin);
    }
    return true;
}

// Each string's encoded length (encode results), one thread per string.
__global__ void encode_results_kernel(const int64_t* __restrict__ src_off, int64_t n,
                                      const __grid_constant__ BatchTables tabs,
                                      const uint8_t* __restrict__ alph_id,
                                      int64_t* __restrict__ results) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int a = alph_id ? (alph_id[i] & (kMaxAlphabets - 1)) : 0;
    results[i] = int64_t(enc_length(uint64_t(src_off[i + 1] - src_off[i]), tabs.padded[a]));
}

// ------------------------------------------------------------------ encode tiles
template <int U>
__global__ void __launch_bounds__(TileShape<U, false>::kThreads)
    encode_batch_kernel(const uint8_t* __restrict__ src, const int64_t* __restrict__ src_off,
                        int64_t n, uint8_t* __restrict__ dst, const int64_t* __restrict__ dst_off,
                        const __grid_constant__ BatchTables tabs,
                        const uint8_t* __restrict__ alph_id) {
    using Sh = TileShape<U, false>;
    constexpr int kWarps = Sh::kWarps, kThreads = Sh::kThreads, S = Sh::kStages;
    constexpr uint32_t T = Sh::T, SIN = Sh::SIN, SOUT = Sh::SOUT;
    extern __shared__ __align__(16) uint8_t smem[];  // [warp][stage] inputs, then [warp] outputs
    __shared__ __align__(16) uint8_t luts[kMaxAlphabets][64];
    __shared__ uint64_t bars[kWarps][S];
    __shared__ Tile ring[kWarps][S];
    __shared__ uint32_t ring_copy[kWarps][S];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < kMaxAlphabets * 16; i += kThreads)
        reinterpret_cast<uint32_t*>(luts)[i] = tabs.enc[i / 16].w[i % 16];
    if (lane == 0) {
        for (int k = 0; k < S; ++k) mbar_init(&bars[warp][k], 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint8_t* sin_base = smem + size_t(warp) * S * SIN;
    uint8_t* sout = smem + size_t(kWarps) * S * SIN + size_t(warp) * SOUT;

    const int64_t origin = src_off[0], bytes = src_off[n] - origin;
    const int64_t GW = int64_t(gridDim.x) * kWarps;
    const int64_t gw = int64_t(blockIdx.x) * kWarps + warp;
    if (bytes <= 0) return;
    const int64_t x0 = origin + bytes * gw / GW, x1 = origin + bytes * (gw + 1) / GW;
    Cursor<false> cur{0, round_boundary<false>(src_off, n, x0, lane),
                      gw + 1 == GW ? src_off[n] : round_boundary<false>(src_off, n, x1, lane)};
    if (cur.pos >= cur.end) return;
    cur.s = cur.pos < src_off[n] ? warp_find_string(src_off, n, cur.pos, lane) : n;
    const uint64_t src_end = uint64_t(src_off[n]);

    auto process = [&](const Tile& t, const uint8_t* sin) {
        const uint64_t a = uint64_t(t.a), b = uint64_t(t.b);
        const bool last = t.b == t.s1;
        const int ai = int(t.id);
        const uint8_t* lut = luts[ai];
        const uint32_t nbytes = uint32_t(b - a);
        const uint32_t triples = nbytes / 3;
        const uint32_t delta = uint32_t((reinterpret_cast<uintptr_t>(src + a)) & 15);
        const uint32_t sh = delta & 3;
        if (nbytes == T) {  // a whole tile: every unit is whole, no tests
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t j = lane + 32 * u;
                const uint4 x = load16_shifted(sin, delta + 12 * j, sh);
                reinterpret_cast<uint4*>(sout)[j] = encode12(x.x, x.y, x.z, lut);
            }
        } else {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t j = lane + 32 * u;
                if (4 * j + 4 <= triples) {
                    const uint4 x = load16_shifted(sin, delta + 12 * j, sh);
                    reinterpret_cast<uint4*>(sout)[j] = encode12(x.x, x.y, x.z, lut);
                } else if (4 * j < triples) {
                    for (uint32_t q = 4 * j; q < triples; ++q) {
                        const uint32_t p = delta + 3 * q;
                        const uint32_t s1b = sin[p], s2b = sin[p + 1], s3b = sin[p + 2];
                        reinterpret_cast<uint32_t*>(sout)[q] =
                            encode_gathered(s2b | (s1b << 8) | (s3b << 16) | (s2b << 24), lut);
                    }
                }
            }
        }
        uint32_t nout = 4 * triples;
        const uint32_t r = nbytes - 3 * triples;  // only the string's last tile has r != 0
        if (last && r) {
            if (lane == 0) {
                const uint32_t p = delta + 3 * triples;
                const uint32_t s1b = sin[p], s2b = r == 2 ? sin[p + 1] : 0u;
                const uint32_t g = s2b | (s1b << 8) | (s2b << 24);
                sout[nout] = lut[(g >> 10) & 63u];
                sout[nout + 1] = lut[(g >> 4) & 63u];
                if (r == 2) sout[nout + 2] = lut[(g >> 22) & 63u];
                if (tabs.padded[ai]) {
                    sout[nout + 3] = '=';
                    if (r == 1) sout[nout + 2] = '=';
                }
            }
            nout += tabs.padded[ai] ? 4 : r + 1;
        }
        __syncwarp();
        const uint64_t rel = a - uint64_t(t.s0);  // a multiple of 3
        warp_stage_out(dst + t.d0 + rel / 3 * 4, sout, nout, lane);
        __syncwarp();  // sout is rewritten by the next tile
    };
    if (!walk_tiles<false, S>(cur, src, src_off, dst_off, alph_id, n, T, src_end, sin_base, SIN,
                              bars[warp], ring[warp], ring_copy[warp], lane, process)) {
        if (lane == 0) atomicOr(&g_fault, 1u);
    }
}

// ------------------------------------------------------------------ decode tiles
template <int U>
__global__ void __launch_bounds__(TileShape<U, true>::kThreads)
    decode_batch_kernel(const uint8_t* __restrict__ src, const int64_t* __restrict__ src_off,
                        int64_t n, uint8_t* __restrict__ dst, const int64_t* __restrict__ dst_off,
                        const __grid_constant__ BatchTables tabs,
                        const uint8_t* __restrict__ alph_id,
                        unsigned long long* __restrict__ err) {
    using Sh = TileShape<U, true>;
    constexpr int kWarps = Sh::kWarps, kThreads = Sh::kThreads, S = Sh::kStages;
    constexpr uint32_t T = Sh::T, SIN = Sh::SIN, SOUT = Sh::SOUT;
    extern __shared__ __align__(16) uint8_t smem[];  // [warp][stage] inputs, then [warp] outputs
    __shared__ __align__(16) uint8_t luts[kMaxAlphabets][256];
    __shared__ uint64_t bars[kWarps][S];
    __shared__ Tile ring[kWarps][S];
    __shared__ uint32_t ring_copy[kWarps][S];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < kMaxAlphabets * 64; i += kThreads)
        reinterpret_cast<uint32_t*>(luts)[i] = tabs.dec[i / 64].w[i % 64];
    if (lane == 0) {
        for (int k = 0; k < S; ++k) mbar_init(&bars[warp][k], 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint8_t* sin_base = smem + size_t(warp) * S * SIN;
    uint8_t* sout = smem + size_t(kWarps) * S * SIN + size_t(warp) * SOUT;

    const int64_t origin = src_off[0], bytes = src_off[n] - origin;
    const int64_t GW = int64_t(gridDim.x) * kWarps;
    const int64_t gw = int64_t(blockIdx.x) * kWarps + warp;
    if (bytes <= 0) return;
    const int64_t x0 = origin + bytes * gw / GW, x1 = origin + bytes * (gw + 1) / GW;
    Cursor<true> cur{0, round_boundary<true>(src_off, n, x0, lane),
                     gw + 1 == GW ? src_off[n] : round_boundary<true>(src_off, n, x1, lane)};
    if (cur.pos >= cur.end) return;
    cur.s = cur.pos < src_off[n] ? warp_find_string(src_off, n, cur.pos, lane) : n;
    const uint64_t src_end = uint64_t(src_off[n]);

    auto process = [&](const Tile& t, const uint8_t* sin) {
        const uint64_t a = uint64_t(t.a), b = uint64_t(t.b);
        const uint8_t* lut = luts[t.id];
        const uint32_t nchars = uint32_t(b - a);  // a multiple of 4
        const uint32_t delta = uint32_t((reinterpret_cast<uintptr_t>(src + a)) & 15);
        uint64_t first = kNoError;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t j = lane + 32 * u;
            if (16 * j + 16 <= nchars) {
                const uint4 c = load16_shifted_u(sin, delta + 16 * j);
                uint32_t e = 0;
                const uint3 o = pack4x24(decode4(c.x, lut, e), decode4(c.y, lut, e),
                                         decode4(c.z, lut, e), decode4(c.w, lut, e));
                uint32_t* ow = reinterpret_cast<uint32_t*>(sout + 12 * j);
                ow[0] = o.x;
                ow[1] = o.y;
                ow[2] = o.z;
                if (e & kBad) {
                    for (uint32_t i = 0; i < 16; ++i) {
                        if (lut[sin[delta + 16 * j + i]] & kBad) {
                            const uint64_t off = a - uint64_t(t.s0) + 16 * j + i;
                            first = off < first ? off : first;
                            break;
                        }
                    }
                }
            } else if (16 * j < nchars) {
                for (uint32_t q = 4 * j; q < nchars / 4; ++q) {
                    const uint32_t p = delta + 4 * q;
                    const uint32_t w = uint32_t(sin[p]) | (uint32_t(sin[p + 1]) << 8) |
                                       (uint32_t(sin[p + 2]) << 16) | (uint32_t(sin[p + 3]) << 24);
                    uint32_t e = 0;
                    const uint32_t v = decode4(w, lut, e);
                    sout[3 * q] = uint8_t(v >> 16);
                    sout[3 * q + 1] = uint8_t(v >> 8);
                    sout[3 * q + 2] = uint8_t(v);
                    if (e & kBad) {
                        for (uint32_t i = 0; i < 4; ++i) {
                            if (lut[sin[p + i]] & kBad) {
                                const uint64_t off = a - uint64_t(t.s0) + 4 * q + i;
                                first = off < first ? off : first;
                                break;
                            }
                        }
                    }
                }
            }
        }
        if (__any_sync(0xffffffffu, first != kNoError)) {  // rare: a bad byte in the tile
            const uint64_t wmin = warp_min_u64(first);
            if (lane == 0) atomicMin(&err[t.s], (unsigned long long)wmin);
        }
        __syncwarp();
        const uint64_t rel = a - uint64_t(t.s0);  // a multiple of 4
        warp_stage_out(dst + t.d0 + rel / 4 * 3, sout, nchars / 4 * 3, lane);
        __syncwarp();  // sout is rewritten by the next tile
    };
    if (!walk_tiles<true, S>(cur, src, src_off, dst_off, alph_id, n, T, src_end, sin_base, SIN,
                             bars[warp], ring[warp], ring_copy[warp], lane, process)) {
        if (lane == 0) atomicOr(&g_fault, 1u);
    }
}

// One thread per string: padding and length rules on the string's tail, its
// bytes, and its result (length or -(offset+1), offset within the string).
__global__ void decode_batch_finalize_kernel(const uint8_t* __restrict__ src,
                                             const int64_t* __restrict__ src_off, int64_t n,
                                             uint8_t* __restrict__ dst,
                                             const int64_t* __restrict__ dst_off,
                                             const __grid_constant__ BatchTables tabs,
                                             const uint8_t* __restrict__ alph_id,
                                             const unsigned long long* __restrict__ err,
                                             int64_t* __restrict__ results) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint8_t* p = src + src_off[i];
    const uint64_t m = uint64_t(src_off[i + 1] - src_off[i]);
    const int ai = alph_id ? (alph_id[i] & (kMaxAlphabets - 1)) : 0;
    const int padded = tabs.padded[ai];
    const uint8_t* tab = reinterpret_cast<const uint8_t*>(tabs.dec[ai].w);
    const uint64_t body = dec_body_length(m);
    uint64_t e = err[i];
    const uint32_t last = m >= 1 ? p[m - 1] : 0u;
    uint32_t pads = 0;
    if (padded && m >= 1 && last == '=') pads = (m >= 2 && p[m - 2] == '=') ? 2 : 1;
    uint32_t v[5] = {0, 0, 0, 0, 0};
    const uint32_t tail = uint32_t(m - body);
    for (uint32_t k = 0; k < tail; ++k) {
        const uint64_t pos = body + k;
        const uint32_t ch = p[pos];
        v[k] = tab[ch];
        if (v[k] & kBad) {
            const bool pad_ok =
                padded && ch == '=' && (pos == m - 1 || (pos + 2 == m && last == '='));
            if (!pad_ok) {
                e = pos < e ? pos : e;
                break;
            }
        }
    }
    if (padded ? (m % 4 != 0) : (m % 4 == 1)) e = m < e ? m : e;
    const uint32_t d = tail - pads;
    if (tabs.canonical[ai] && (d % 4 == 2 || d % 4 == 3)) {
        // the last data character's bits that reach no output byte must be zero
        const uint32_t last_v = v[d - 1], low = d % 4 == 2 ? 15u : 3u;
        const uint64_t pos = body + d - 1;
        if (!(last_v & kBad) && (last_v & low)) e = pos < e ? pos : e;
    }
    if (e != kNoError) {
        results[i] = -int64_t(e) - 1;
        return;
    }
    uint8_t* q = dst + dst_off[i];
    uint64_t o = body / 4 * 3;
    for (uint32_t j = 0; j < d; j += 4) {
        const uint32_t k = d - j < 4 ? d - j : 4;
        const uint32_t a = v[j], bb = k > 1 ? v[j + 1] : 0u, c = k > 2 ? v[j + 2] : 0u,
                       dd = k > 3 ? v[j + 3] : 0u;
        const uint32_t w = ((a * 64u + bb) * 64u + c) * 64u + dd;
        const uint32_t nb = k == 4 ? 3u : k - 1;
        for (uint32_t t = 0; t < nb; ++t) q[o++] = uint8_t(w >> (16 - 8 * t));
    }
    results[i] = int64_t(o);
}

struct Occ {
    std::once_flag once;
    cudaError_t err = cudaSuccess;
    int ctas = 1;
};

// Allows the kernel up to max_smem bytes of dynamic shared memory and
// returns its resident blocks per SM with smem bytes (once per kernel,
// device and smem).
template <class K>
int occupancy(K kernel, int threads, size_t smem, size_t max_smem, Occ& occ, cudaError_t* err) {
    std::call_once(occ.once, [&] {
        if (max_smem > 48 * 1024)
            occ.err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           int(max_smem));
        int c = 1;
        if (occ.err == cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, kernel, threads, smem) != cudaSuccess)
            c = 1;
        occ.ctas = c > 0 ? c : 1;
    });
    *err = occ.err;
    return occ.ctas;
}

Occ g_enc_occ[4][64], g_dec_occ[4][64];

int unit_slot(int units) { return units == 1 ? 0 : units == 2 ? 1 : units == 4 ? 2 : 3; }

template <int U>
cudaError_t launch_encode_tiles(const BatchArgs& a, const BatchTables& t, cudaStream_t st) {
    using Sh = TileShape<U, false>;
    const DeviceInfo& di = device_info();
    cudaError_t e = cudaSuccess;
    const int occ = occupancy(encode_batch_kernel<U>, Sh::kThreads, Sh::kSmem, Sh::kSmem,
                              g_enc_occ[unit_slot(U)][di.device & 63], &e);
    if (e != cudaSuccess) return e;
    encode_batch_kernel<U><<<unsigned(di.sm_count * occ), Sh::kThreads, Sh::kSmem, st>>>(
        a.src, a.src_off, a.n, a.dst, a.dst_off, t, a.alph_id);
    return cudaGetLastError();
}

template <int U>
cudaError_t launch_decode_tiles(const BatchArgs& a, const BatchTables& t,
                                unsigned long long* err, cudaStream_t st) {
    using Sh = TileShape<U, true>;
    const DeviceInfo& di = device_info();
    cudaError_t e = cudaSuccess;
    const int occ = occupancy(decode_batch_kernel<U>, Sh::kThreads, Sh::kSmem, Sh::kSmem,
                              g_dec_occ[unit_slot(U)][di.device & 63], &e);
    if (e != cudaSuccess) return e;
    decode_batch_kernel<U><<<unsigned(di.sm_count * occ), Sh::kThreads, Sh::kSmem, st>>>(
        a.src, a.src_off, a.n, a.dst, a.dst_off, t, a.alph_id, err);
    return cudaGetLastError();
}

// Inclusive scan over the warp's lanes.
__device__ __forceinline__ int64_t warp_inclusive_scan(int64_t v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// dst_off = exclusive scan of per-string output capacities, in three
// launches and no workspace:
//   1. block b scans its kOffItems strings (kOffThreads threads x kScanItems
//      each) and writes their block-local exclusive offsets, except that the
//      block's first slot (local offset 0) receives the block's total;
//   2. one block turns those totals into block prefixes in place (and writes
//      dst_off[n], the grand total);
//   3. block b adds its prefix (its first slot, now final) to its other slots.
constexpr int kScanItems = 8;
constexpr int kOffThreads = 256;
constexpr int64_t kOffItems = int64_t(kOffThreads) * kScanItems;  // strings per block

template <bool kDecode>
__device__ __forceinline__ int64_t capacity(const int64_t* __restrict__ src_off, int64_t i,
                                            const BatchTables& tabs,
                                            const uint8_t* __restrict__ alph_id) {
    const uint64_t len = uint64_t(src_off[i + 1] - src_off[i]);
    if (kDecode) return int64_t((len + 3) / 4 * 3);
    const int al = alph_id ? (alph_id[i] & (kMaxAlphabets - 1)) : 0;
    return int64_t(enc_length(len, tabs.padded[al]));
}

template <bool kDecode>
__global__ void __launch_bounds__(kOffThreads)
    offsets_local_kernel(const int64_t* __restrict__ src_off, int64_t n,
                         const __grid_constant__ BatchTables tabs,
                         const uint8_t* __restrict__ alph_id, int64_t* __restrict__ dst_off) {
    __shared__ int64_t warp_sum[kOffThreads / 32];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t first = int64_t(blockIdx.x) * kOffItems;
    const int64_t i0 = first + int64_t(tid) * kScanItems;
    int64_t cap[kScanItems], sum = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        cap[j] = i0 + j < n ? capacity<kDecode>(src_off, i0 + j, tabs, alph_id) : 0;
        sum += cap[j];
    }
    const int64_t incl = warp_inclusive_scan(sum, lane);
    if (lane == 31) warp_sum[warp] = incl;
    __syncthreads();
    int64_t before = 0, total = 0;
#pragma unroll
    for (int w = 0; w < kOffThreads / 32; ++w) {
        before += w < warp ? warp_sum[w] : 0;
        total += warp_sum[w];
    }
    int64_t run = before + incl - sum;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        if (i0 + j < n) dst_off[i0 + j] = (i0 + j == first) ? total : run;
        run += cap[j];
    }
}

// One block: dst_off[b * kOffItems] (block totals) -> block prefixes; dst_off[n].
__global__ void __launch_bounds__(1024)
    offsets_blocks_kernel(int64_t n, int64_t* __restrict__ dst_off) {
    __shared__ int64_t warp_sum[32];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t nblk = (n + kOffItems - 1) / kOffItems;
    int64_t carry = 0;
    for (int64_t base = 0; base < nblk; base += 1024) {
        const int64_t b = base + tid;
        const int64_t t = b < nblk ? dst_off[b * kOffItems] : 0;
        const int64_t incl = warp_inclusive_scan(t, lane);
        if (lane == 31) warp_sum[warp] = incl;
        __syncthreads();
        int64_t before = 0, total = 0;
        for (int w = 0; w < 32; ++w) {
            before += w < warp ? warp_sum[w] : 0;
            total += warp_sum[w];
        }
        if (b < nblk) dst_off[b * kOffItems] = carry + before + incl - t;
        carry += total;
        __syncthreads();  // warp_sum is rewritten by the next round
    }
    if (tid == 0) dst_off[n] = carry;
}

__global__ void __launch_bounds__(kOffThreads)
    offsets_fix_kernel(int64_t n, int64_t* __restrict__ dst_off) {
    const int64_t first = int64_t(blockIdx.x) * kOffItems;
    const int64_t prefix = dst_off[first];
    for (int64_t i = first + 1 + threadIdx.x; i < first + kOffItems && i < n; i += kOffThreads)
        dst_off[i] += prefix;
}

}  // namespace

uint32_t batch_fault_flag(bool clear) {
    uint32_t v = 0;
    cudaMemcpyFromSymbol(&v, g_fault, sizeof(v));
    if (clear && v) {
        const uint32_t z = 0;
        cudaMemcpyToSymbol(g_fault, &z, sizeof(z));
    }
    return v;
}

size_t batch_workspace_bytes(int64_t n) {
    // One error word per string (decode).
    return size_t(n) * sizeof(uint64_t);
}

cudaError_t launch_batch(bool decode, const BatchArgs& a, const BatchTables& tabs, int units,
                         void* workspace, cudaStream_t st) {
    if (!decode) {
        encode_results_kernel<<<unsigned((a.n + 255) / 256), 256, 0, st>>>(a.src_off, a.n, tabs,
                                                                           a.alph_id, a.results);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        switch (units) {
            case 1: return launch_encode_tiles<1>(a, tabs, st);
            case 2: return launch_encode_tiles<2>(a, tabs, st);
            case 4: return launch_encode_tiles<4>(a, tabs, st);
            default: return launch_encode_tiles<8>(a, tabs, st);
        }
    }
    unsigned long long* err = static_cast<unsigned long long*>(workspace);
    cudaError_t e = cudaMemsetAsync(err, 0xFF, size_t(a.n) * sizeof(uint64_t), st);  // kNoError
    if (e != cudaSuccess) return e;
    switch (units) {
        case 1: e = launch_decode_tiles<1>(a, tabs, err, st); break;
        case 2: e = launch_decode_tiles<2>(a, tabs, err, st); break;
        case 4: e = launch_decode_tiles<4>(a, tabs, err, st); break;
        default: e = launch_decode_tiles<8>(a, tabs, err, st); break;
    }
    if (e != cudaSuccess) return e;
    const unsigned grid = unsigned((a.n + 255) / 256);
    decode_batch_finalize_kernel<<<grid, 256, 0, st>>>(a.src, a.src_off, a.n, a.dst, a.dst_off,
                                                       tabs, a.alph_id, err, a.results);
    return cudaGetLastError();
}

}  // namespace b64

namespace b64 {

cudaError_t launch_batch_offsets(bool decode, const int64_t* src_off, int64_t n,
                                 const BatchTables& tabs, const uint8_t* alph_id,
                                 int64_t* dst_off, cudaStream_t st) {
    const unsigned nblk = unsigned((n + kOffItems - 1) / kOffItems);
    if (nblk) {
        if (decode)
            offsets_local_kernel<true><<<nblk, kOffThreads, 0, st>>>(src_off, n, tabs, alph_id,
                                                                     dst_off);
        else
            offsets_local_kernel<false><<<nblk, kOffThreads, 0, st>>>(src_off, n, tabs, alph_id,
                                                                      dst_off);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    offsets_blocks_kernel<<<1, 1024, 0, st>>>(n, dst_off);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || nblk == 0) return e;
    offsets_fix_kernel<<<nblk, kOffThreads, 0, st>>>(n, dst_off);
    return cudaGetLastError();
}

}  // namespace b64
