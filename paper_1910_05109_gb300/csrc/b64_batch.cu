// Batched variable-length encode and strict decode: many independent strings
// in one persistent launch (the paper's codec, Sec. 3.1 and Sec. 3.2, applied
// per string; batching itself is not in the paper).
//
// String i is src[src_off[i] .. src_off[i+1]) and goes to dst + dst_off[i],
// with its own alphabet (one of up to kMaxAlphabets passed by value). A warp
// codes a tile of 32 x U units of 12 input bytes (encode) or 16 characters
// (decode) at a time, U chosen at launch (the autotuner's tile size).
//
// Launch sequence (all on one stream, so it can be recorded in a CUDA graph):
//   1. encode: one thread per string writes the string's output length to
//      results; decode: the per-string error words in the caller's workspace
//      are set to "none" (a memset);
//   2. tile kernel (persistent, 8-warp blocks): the concatenated
//      input is split into equal byte ranges, one per warp. A warp finds the
//      strings that hold its range ends with a 32-way search over src_off and
//      moves both ends up to the next 3-byte (encode) or 4-character (decode)
//      group boundary of their string, so neighbouring warps meet without
//      talking to each other and no per-string scan is needed. Within its
//      range a string's part is cut into units of 12 bytes (encode) or 16
//      characters (decode), the last one possibly shorter. The warp walks its
//      range in tiles of TB consecutive unit start positions; a tile's bytes
//      come into the warp's shared-memory ring by one bulk (TMA) copy, the
//      next tiles' copies started before the current one is coded (or aligned
//      loads where the span would leave the source buffer). The strings are
//      known from a window of 32 strings' metadata (their units counted by a
//      warp scan). A whole tile of full units of one string runs as one
//      unrolled block, U units a lane with uniform addressing. Other tiles
//      go in rounds: where every string with units in the round has its
//      output aligned for a unit's stores (16 bytes encode, 4 decode;
//      b64_batch_offsets' B64_OFFSETS_ALIGN16 layout gives every string
//      that), a mixed round codes consecutive units of whichever strings
//      hold them, V a lane when the tile has 32 V units left (so that each
//      lane has independent units in flight), else one a lane, each lane
//      finding its units' strings from the strings that start inside the
//      round, and stores them straight from registers; otherwise a string's
//      units in the tile (a piece) go in rounds of 32 with uniform
//      addressing, and an unaligned string's output is appended to a
//      pending run in shared memory, written out with aligned 16-byte stores
//      once the run breaks, fills, or ends past a string's last unit. A
//      string's short last unit is finished by its lane with the padding
//      rules. Decode rounds fold bad-byte offsets into the string's error
//      word with an atomic minimum;
//   3. decode only: one thread per string applies the padding and length
//      rules to the string's last 2..5 characters and writes its result.
#include <mutex>
#include <type_traits>

// The batched encoder is bound by the ALU pipe with the FMA pipe mostly idle:
// its middle 6-bit fields are taken with a multiply and a multiply-high and
// its characters joined by multiply-adds (both on the FMA pipe), which
// measured 199 -> 170 us on 100,000 strings (aligned outputs), 251 -> 231 us
// (packed). Still selectable with -D for comparison.
#ifndef B64_ENC_VARIANT
#define B64_ENC_VARIANT 2
#endif
#ifndef B64_JOIN_WITH_PRMT
#define B64_JOIN_WITH_PRMT 0
#endif

#include "b64_internal.h"
#include "b64_smem.cuh"

namespace b64 {
namespace {


#ifndef B64_BATCH_STAGES
#define B64_BATCH_STAGES 3
#endif
// The widest tiles (U = 8) take two stages and at most 128 registers a
// thread, so that two blocks fit an SM (with three stages one block's shared
// memory is over half an SM's; measured: two blocks code the 100k-string
// batch about 28% faster than one, in both directions).
#ifndef B64_BATCH_WIDE_STAGES
#define B64_BATCH_WIDE_STAGES 2
#endif
// Rounds that mix strings, where every string in them is stored from
// registers (0: a round never mixes strings).
#ifndef B64_BATCH_MIXED
#define B64_BATCH_MIXED 1
#endif
// Units a lane in a wide mixed round of the decoder with 8-unit tiles (1 to
// 4; narrower tiles take at most 2). Wide rounds measured 187 -> 179 us on
// 100,000 strings with aligned outputs; the encoder's measured slower (its
// rounds stay one unit a lane).
#ifndef B64_BATCH_MIXED_UNITS
#define B64_BATCH_MIXED_UNITS 4
#endif
// How far the whole-tile loop over its U units a lane is unrolled (decoder,
// encoder): a smaller kernel measured faster for the decoder on 100,000
// strings (8 -> 2: 179 -> 174 us), where the mixed rounds' code competes for
// the instruction cache.
#ifndef B64_BATCH_DEC_WHOLE_UNROLL
#define B64_BATCH_DEC_WHOLE_UNROLL 2
#endif
#ifndef B64_BATCH_ENC_WHOLE_UNROLL
#define B64_BATCH_ENC_WHOLE_UNROLL 8
#endif
#ifndef B64_BATCH_WIDE_MIN_BLOCKS
#define B64_BATCH_WIDE_MIN_BLOCKS 2
#endif

// The tile kernels' shape for tiles of 32 x U units: 8 warps a block, as many
// blocks an SM as fit (three for U <= 4, two for U = 8); each warp has a ring of kStages staging buffers
// (kStages - 1 tiles in flight while one is coded) and a buffer for its
// pending output run, in dynamic shared memory. A staging buffer holds a
// tile's span: up to TB + G - 1 bytes, 15 more on each side for 16-byte
// alignment, and slack for a unit's word reads past its last byte.
template <int U, bool kDecode>
struct TileShape {
    static constexpr int kWarps = 8;
    // blocks an SM the registers allow
    static constexpr int kMinBlocks = U >= 8 ? B64_BATCH_WIDE_MIN_BLOCKS : 3;
    static constexpr int kThreads = 32 * kWarps;
    static constexpr int kStages = U >= 8 ? B64_BATCH_WIDE_STAGES : B64_BATCH_STAGES;
    static constexpr uint32_t G = kDecode ? 16 : 12;        // input bytes of a full unit
    static constexpr uint32_t O = kDecode ? 12 : 16;        // output bytes of a full unit
    static constexpr uint32_t TB = 32 * U * G;              // unit start positions per tile
    static constexpr uint32_t SIN = (TB + G + 48 + 15) & ~15u;
    static constexpr uint32_t RUN = 32 * U * O;             // pending-run capacity
    static constexpr uint32_t SOUT = RUN + 32;              // + the copy-out's read slack
    static constexpr size_t kSmem = size_t(kWarps) * (size_t(kStages) * SIN + SOUT);
    static_assert(SIN % 16 == 0 && RUN % 16 == 0 && kStages >= 2 && kStages <= 8, "shape");
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
// rounded up to the next unit boundary (12 bytes for encode, 16 characters
// for decode, counted from the start of the string that holds x), but not
// past the end of the string's coded part (its end; for decode, its body).
// Every warp rounds the same way, so neighbouring ranges meet exactly, and a
// segment's output starts a multiple of 16 (encode) or 12 (decode) bytes
// into its string's output.
template <bool kDecode>
__device__ __forceinline__ int64_t round_boundary(const int64_t* __restrict__ src_off, int64_t n,
                                                  int64_t x, int lane) {
    if (x >= src_off[n]) return src_off[n];
    const int64_t s = warp_find_string(src_off, n, x, lane);
    const int64_t s0 = src_off[s];
    const int64_t len = src_off[s + 1] - s0;
    const int64_t lim = kDecode ? int64_t(dec_body_length(uint64_t(len))) : len;
    constexpr int64_t g = kDecode ? 16 : 12;  // whole units: a unit never spans two warps
    const int64_t r = (x - s0 + g - 1) / g * g;
    return s0 + (r < lim ? r : lim);
}

// ------------------------------------------------------------------ string window
// The metadata of 32 consecutive strings w0 .. w0 + 31, one string a lane,
// as their parts in the warp's range [P0, end): the segment [seg_lo, seg_hi)
// of string i is its coded part (encode: all of it; decode: all but its last
// 2..5 characters) clipped to the range. Each segment is cut into units of G
// bytes (the last one possibly shorter); units are numbered through the
// warp's range in order, so a segment's units are us .. us + un - 1.
// Positions are kept relative to P0 (a warp's range is far below 4 GiB). The
// lane that holds a string keeps its counts in registers (for the ballots)
// and writes the rest to the warp's record in shared memory, where every
// lane reads the record of the string it works on.
struct WinRec {
    int64_t dst[32];  // where the segment's output starts (dst offset)
    int64_t rel[32];  // segment start within its string (decode error offsets)
    uint32_t lo[32];  // segment start, relative to P0
    uint32_t us[32];  // first unit
    uint32_t un[32];  // units
    uint32_t fl[32];  // bytes of the last unit | alphabet << 8 | padded << 16
    uint8_t slot[32 * B64_BATCH_MIXED_UNITS];  // mixed rounds: the string starting at unit R + d
};

struct Win {
    int64_t w0;       // first string of the window
    int64_t next;     // where string w0 + 32 starts, relative to P0 (src_off[min(w0 + 32, n)])
    uint32_t lo;      // this lane's string: segment start (relative to P0)
    uint32_t us, un;  // this lane's string: first unit, units
    uint32_t base;    // units of the warp's range before the window
    uint32_t end_u;   // units up to the window's end
    uint32_t dirm;    // bit i: string w0 + i's segment output is aligned for a unit's stores
};

template <bool kDecode, uint32_t G, uint32_t A>
__device__ __forceinline__ void load_window(Win& w, WinRec& r, int64_t s, uint32_t base,
                                            const int64_t* __restrict__ src_off,
                                            const uint8_t* dst,
                                            const int64_t* __restrict__ dst_off,
                                            const uint8_t* __restrict__ alph_id,
                                            const BatchTables& tabs, int64_t n, int64_t P0,
                                            int64_t end, int lane) {
    __syncwarp();  // every lane is done with the previous window's records
    const int64_t i = s + lane;
    const bool valid = i < n;
    int64_t lo = 0, hi = 0, d = 0;
    uint32_t id = 0;
    if (valid) {
        lo = src_off[i];
        hi = src_off[i + 1];
        d = dst_off[i];
        id = alph_id ? uint32_t(alph_id[i] & (kMaxAlphabets - 1)) : 0u;
    }
    const int64_t lim = lo + (kDecode ? int64_t(dec_body_length(uint64_t(hi - lo))) : hi - lo);
    const int64_t sl = lo > P0 ? lo : P0;
    const int64_t sh = lim < end ? lim : end;
    const uint32_t nb = (valid && sh > sl) ? uint32_t(sh - sl) : 0u;
    const uint32_t un = (nb + G - 1) / G;
    uint32_t incl = un;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    w.w0 = s;
    w.base = base;
    w.us = base + incl - un;
    w.un = un;
    w.lo = uint32_t(sl - P0);
    w.end_u = base + __shfl_sync(0xffffffffu, incl, 31);
    w.next = src_off[s + 32 < n ? s + 32 : n] - P0;
    r.lo[lane] = w.lo;
    const int64_t seg_dst = d + (kDecode ? (sl - lo) / 4 * 3 : (sl - lo) / 3 * 4);
    r.dst[lane] = seg_dst;
    w.dirm = __ballot_sync(0xffffffffu,
                           un == 0 || ((reinterpret_cast<uintptr_t>(dst) + uint64_t(seg_dst)) &
                                       (A - 1)) == 0);
    r.rel[lane] = sl - lo;
    r.us[lane] = w.us;
    r.un[lane] = un;
    const uint32_t nbl = un ? nb - (un - 1) * G : 0u;
    r.fl[lane] = nbl | (id << 8) | (tabs.padded[id] ? 1u << 16 : 0u);
    __syncwarp();
}

// Units of the window whose start lies below position q (relative to P0).
template <uint32_t G>
__device__ __forceinline__ uint32_t units_below(const Win& w, uint32_t q) {
    uint32_t c = 0;
    if (w.un > 0 && q > w.lo) {
        const uint32_t u = (q - w.lo + G - 1) / G;
        c = u < w.un ? u : w.un;
    }
    return w.base + __reduce_add_sync(0xffffffffu, c);
}

// Bytes b .. 3 of word w cleared (b <= 0: all of them).
__device__ __forceinline__ uint32_t keep_bytes(uint32_t w, int b) {
    return b >= 4 ? w : (b <= 0 ? 0u : (w & ((1u << (8 * b)) - 1u)));
}

// A string's last unit when it is shorter than a whole one: nb (1..11)
// bytes in x (bytes past them read as zero, Sec. 2: a partial final group is
// completed with zero bits), coded with the string's padding rule. Returns
// the characters; *nout = their count.
__device__ __forceinline__ uint4 pad_last_unit(uint4 ch, uint32_t nb, bool padded,
                                               uint32_t* nout) {
    const uint32_t t3 = nb / 3, r = nb - 3 * t3;
    *nout = 4 * t3 + (r == 0 ? 0u : padded ? 4u : r + 1);
    if (r && padded) {  // '=' after the last group's characters
        const uint32_t m = r == 1 ? 0x0000FFFFu : 0x00FFFFFFu;
        const uint32_t pad = r == 1 ? 0x3D3D0000u : 0x3D000000u;
        if (t3 == 0) ch.x = (ch.x & m) | pad;
        else if (t3 == 1) ch.y = (ch.y & m) | pad;
        else if (t3 == 2) ch.z = (ch.z & m) | pad;
        else ch.w = (ch.w & m) | pad;
    }
    return ch;
}
__device__ __forceinline__ uint4 encode_last_unit(uint4 x, uint32_t nb, bool padded,
                                                  const uint8_t* lut, uint32_t* nout) {
    const uint4 ch = encode12(keep_bytes(x.x, int(nb)), keep_bytes(x.y, int(nb) - 4),
                              keep_bytes(x.z, int(nb) - 8), lut);
    return pad_last_unit(ch, nb, padded, nout);
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

// The 16 staged characters at sbuf[off ..] of a decode unit: three 64-bit
// loads from the 8-byte boundary at or below off, one level of selects for
// off mod 8 >= 4, then funnel shifts for off mod 4. Lanes may differ in off.
// (Measured on the 100k-string decode against two 128-bit loads with a
// four-way choice of words: 190 -> 184 us; five 32-bit loads, whose
// lanes meet four to a bank, 186 us.) Reads up to 24 bytes from off & ~7.
__device__ __forceinline__ uint4 load_unit16(const uint8_t* sbuf, uint32_t off) {
    const uint32_t A = off & ~7u, sb = 8 * (off & 3u);
    const uint2 a = *reinterpret_cast<const uint2*>(sbuf + A);
    const uint2 b = *reinterpret_cast<const uint2*>(sbuf + A + 8);
    const uint2 c = *reinterpret_cast<const uint2*>(sbuf + A + 16);
    const bool o1 = (off & 4u) != 0;
    const uint32_t v0 = o1 ? a.y : a.x, v1 = o1 ? b.x : a.y, v2 = o1 ? b.y : b.x,
                   v3 = o1 ? c.x : b.y, v4 = o1 ? c.y : c.x;
    return make_uint4(__funnelshift_r(v0, v1, sb), __funnelshift_r(v1, v2, sb),
                      __funnelshift_r(v2, v3, sb), __funnelshift_r(v3, v4, sb));
}

// The first bad byte among the n staged characters at sbuf[o ..] (one is
// known to be there), folded into the string's error word as offset base + i.
// Kept out of line: it is rare, and the hot loops stay smaller.
__device__ __noinline__ void record_first_bad(const uint8_t* sbuf, uint32_t o, uint32_t n,
                                              const uint8_t* lut, unsigned long long* word,
                                              uint64_t base) {
    for (uint32_t i = 0; i < n; ++i)
        if (lut[sbuf[o + i]] & kBad) {
            atomicMin(word, (unsigned long long)(base + i));
            return;
        }
}

// A flag that is a run-time bool in one copy of a loop and a compile-time
// constant (std::true_type / std::false_type) in others.
__device__ __forceinline__ bool flag_value(bool b) { return b; }
template <bool B>
__device__ __forceinline__ constexpr bool flag_value(std::integral_constant<bool, B>) { return B; }

// ------------------------------------------------------------------ tile kernels
// One persistent kernel for both directions (see the file comment).
template <int U, bool kDecode, bool kPairs = false>
__global__ void __launch_bounds__(TileShape<U, kDecode>::kThreads,
                                  TileShape<U, kDecode>::kMinBlocks)
    batch_tile_kernel(const uint8_t* __restrict__ src, const int64_t* __restrict__ src_off,
                      int64_t n, uint8_t* __restrict__ dst, const int64_t* __restrict__ dst_off,
                      const __grid_constant__ BatchTables tabs,
                      const uint8_t* __restrict__ alph_id, unsigned long long* __restrict__ err) {
    using Sh = TileShape<U, kDecode>;
    constexpr int kWarps = Sh::kWarps, kThreads = Sh::kThreads, S = Sh::kStages;
    constexpr uint32_t G = Sh::G, O = Sh::O, TB = Sh::TB, SIN = Sh::SIN, RUN = Sh::RUN,
                       SOUT = Sh::SOUT;
    constexpr uint32_t A = kDecode ? 4u : 16u;  // alignment a unit's output store needs
    constexpr bool kMixed = B64_BATCH_MIXED != 0;
    constexpr int kWholeUnrollSet = kDecode ? B64_BATCH_DEC_WHOLE_UNROLL : B64_BATCH_ENC_WHOLE_UNROLL;
    constexpr int kWholeUnroll = kWholeUnrollSet < U ? kWholeUnrollSet : U;
    // units a lane in a wide mixed round (decode only; at most 2 under the
    // 80-register bound of the narrower tiles)
    constexpr uint32_t V = !kDecode ? 1u
                           : U >= 8 || B64_BATCH_MIXED_UNITS < 2 ? B64_BATCH_MIXED_UNITS : 2u;
    constexpr int LUT = kDecode ? 256 : 64;
    extern __shared__ __align__(16) uint8_t smem[];  // [warp][stage] inputs, then [warp] runs
    __shared__ __align__(256) uint8_t luts[kMaxAlphabets][LUT];
    __shared__ uint64_t bars[kWarps][S];
    __shared__ WinRec recs[kWarps];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < kMaxAlphabets * LUT / 4; i += kThreads)
        reinterpret_cast<uint32_t*>(luts)[i] =
            kDecode ? tabs.dec[i / 64].w[i % 64] : tabs.enc[i / 16].w[i % 16];
    if (lane == 0) {
        for (int k = 0; k < S; ++k) mbar_init(&bars[warp][k], 1);
        fence_mbar_init();
    }
    __syncthreads();
    // encode with pair tables (kPairs): per alphabet the 4096 character pairs
    // of two adjacent 6-bit fields, after the staging and run buffers
    uint16_t* const pairs = reinterpret_cast<uint16_t*>(smem + Sh::kSmem);
    const uint32_t npair = kPairs ? uint32_t(tabs.n_alph) : 0u;
    if constexpr (kPairs) {
        for (uint32_t i = tid; i < npair * 4096u; i += kThreads) {
            const uint8_t* l = luts[i >> 12];
            pairs[i] = uint16_t(uint32_t(l[(i >> 6) & 63u]) | (uint32_t(l[i & 63u]) << 8));
        }
        __syncthreads();
    }
    // 12 bytes -> 16 characters with alphabet id (its byte table lut), in
    // the whole-tile loop (pair tables made whole tiles faster, 144 -> 130 us
    // on 300 strings of 1 MiB, but the kernel's mixed rounds slower even with
    // their byte tables, 165 -> 174 us on 100,000 lognormal strings: the
    // autotuner picks per batch shape)
    auto enc12 = [&](const uint4& x, uint32_t id, const uint8_t* lut) -> uint4 {
        if constexpr (kPairs)
            return encode12_pairs(x.x, x.y, x.z, pairs + ((id < npair ? id : 0u) << 12));
        else
            return encode12(x.x, x.y, x.z, lut);
    };
    uint8_t* const sin_base = smem + size_t(warp) * S * SIN;
    uint8_t* const sout = smem + size_t(kWarps) * S * SIN + size_t(warp) * SOUT;
    WinRec& rec = recs[warp];

    const int64_t origin = src_off[0], bytes = src_off[n] - origin;
    const int64_t GW = int64_t(gridDim.x) * kWarps;
    const int64_t gw = int64_t(blockIdx.x) * kWarps + warp;
    if (bytes <= 0) return;
    const int64_t x0 = origin + bytes * gw / GW, x1 = origin + bytes * (gw + 1) / GW;
    const int64_t P0 = round_boundary<kDecode>(src_off, n, x0, lane);
    const int64_t end = gw + 1 == GW ? src_off[n] : round_boundary<kDecode>(src_off, n, x1, lane);
    if (P0 >= end) return;
    if (end - P0 > int64_t(0x7FFFFFFF)) {  // positions are kept in 32 bits
        if (lane == 0) atomicOr(&g_fault, 2u);
        return;
    }
    const uint32_t span = uint32_t(end - P0);
    const uint32_t ntiles = (span + TB - 1) / TB;
    const uint64_t src_end = uint64_t(src_off[n]);
    const uint8_t* const srcp = src + P0;  // positions below are relative to P0

    Win win;
    load_window<kDecode, G, A>(win, rec, warp_find_string(src_off, n, P0, lane), 0u, src_off,
                               dst, dst_off, alph_id, tabs, n, P0, end, lane);

    // Tile t holds the units that start in [t TB, min((t+1) TB, span)); their
    // bytes end before min(q + G - 1, span). Lane 0 keeps a bit per ring
    // stage: 1 if that stage's tile comes by bulk copy.
    uint32_t copy_bits = 0, phases = 0;
    auto issue = [&](uint32_t t) {
        if (lane == 0) {
            const int k = int(t % S);
            const uint32_t p = t * TB, q = p + TB < span ? p + TB : span;
            const uint32_t b = q + G - 1 < span ? q + G - 1 : span;
            const bool c = issue_tile_load(sin_base + size_t(k) * SIN, src, uint64_t(P0) + p,
                                           uint64_t(P0) + b, src_end, &bars[warp][k]);
            copy_bits = (copy_bits & ~(1u << k)) | (c ? 1u << k : 0u);
        }
    };
    for (uint32_t t = 0; t < S - 1 && t < ntiles; ++t) issue(t);

    uint8_t* run_dst = nullptr;  // the pending run: sout[0 .. run_len) goes to run_dst
    uint32_t run_len = 0;
    auto flush = [&]() {
        __syncwarp();
        warp_stage_out(run_dst, sout, run_len, lane);
        __syncwarp();
        run_len = 0;
    };
    // makes the run end at d with room for `need` bytes and a store-aligned end
    auto run_at = [&](uint8_t* d, uint32_t need) {
        if (run_len && (run_dst + run_len != d || run_len % A != 0 || run_len + need > RUN))
            flush();
        if (run_len == 0) run_dst = d;
    };

    uint32_t R = 0;  // the next unit to code
    for (uint32_t t = 0; t < ntiles; ++t) {
        const int k = int(t % S);
        fence_proxy_async_smem();  // this lane's reads of tile t - 1 before the copy below
        __syncwarp();              // every lane is done with tile t - 1's buffer
        if (t + S - 1 < ntiles) issue(t + S - 1);
        const uint32_t p = t * TB, q = p + TB < span ? p + TB : span;
        const uint32_t b = q + G - 1 < span ? q + G - 1 : span;
        uint8_t* const sin = sin_base + size_t(k) * SIN;
        const bool by_copy = ((__shfl_sync(0xffffffffu, copy_bits, 0) >> k) & 1u) != 0;
        if (!tile_ready(by_copy, sin, &bars[warp][k], phases, k, src, uint64_t(P0) + p,
                        uint64_t(P0) + b, src_end, lane)) {
            // let the copies still in flight land (bounded) before the block can
            // exit; this tile's wait already flipped its parity
            if (lane == 0) {
                for (uint32_t i = t; i < ntiles && i < t + S - 1; ++i) {
                    const int kk = int(i % S);
                    if ((copy_bits >> kk) & 1u)
                        mbar_wait(&bars[warp][kk], ((phases >> kk) & 1u) ^ (i == t ? 1u : 0u));
                }
                atomicOr(&g_fault, 1u);
            }
            return;
        }
        // the byte at position x sits at sin[x - p + delta]
        const uint32_t delta = uint32_t(reinterpret_cast<uintptr_t>(srcp + p) & 15u);
        for (;;) {
            const uint32_t Rq = units_below<G>(win, q);
            if (Rq - R == 32u * U) {
                // ---- a whole tile of full units of one string: one record, U
                //      rounds with uniform addressing and no per-round tests
                const int k0 = 31 - __clz(__ballot_sync(0xffffffffu, win.un > 0 && win.us <= R));
                const int kq =
                    31 - __clz(__ballot_sync(0xffffffffu, win.un > 0 && win.us <= Rq - 1));
                const uint32_t fl0 = rec.fl[k0], us0 = rec.us[k0];
                const uint32_t full0 = rec.un[k0] - ((fl0 & 0xFFu) < G ? 1u : 0u);
                if (k0 == kq && Rq - us0 <= full0) {
                    const uint8_t* lut = luts[(fl0 >> 8) & 0xFFu];
                    const uint32_t j0 = R - us0;
                    const uint32_t o0 = rec.lo[k0] + G * j0 - p + delta;
                    uint8_t* const d0 = dst + rec.dst[k0] + int64_t(O) * j0;
                    // an aligned string output takes each unit's stores straight
                    // from registers; any other goes through the run buffer
                    const bool direct = (reinterpret_cast<uintptr_t>(d0) & (A - 1)) == 0;
                    if (!direct) {
                        if (run_len) flush();
                        run_dst = d0;
                    }
                    // one copy of the loop for each store target (global memory or
                    // the run buffer), so each keeps its own address space
                    auto whole = [&](auto direct_tile) {
                        const bool dd = flag_value(direct_tile);  // a constant in encode's copies
#pragma unroll (kWholeUnroll)
                        for (int u = 0; u < U; ++u) {
                            const uint32_t i = 32 * u + lane;  // unit j0 + i
                            const uint32_t o = o0 + G * i;
                            if constexpr (kDecode) {
                                const uint4 c = load_unit16(sin, o);  // o mod 16 uniform
                                uint32_t e = 0;
                                const uint32_t lb = smem_addr(lut);
                                const uint3 v =
                                    pack4x24(decode4_at(c.x, lb, e), decode4_at(c.y, lb, e),
                                             decode4_at(c.z, lb, e), decode4_at(c.w, lb, e));
                                if (dd) {
                                    uint32_t* ow = reinterpret_cast<uint32_t*>(d0 + 12 * i);
                                    ow[0] = v.x;
                                    ow[1] = v.y;
                                    ow[2] = v.z;
                                } else {
                                    uint32_t* ow = reinterpret_cast<uint32_t*>(sout + 12 * i);
                                    ow[0] = v.x;
                                    ow[1] = v.y;
                                    ow[2] = v.z;
                                }
                                if (e & kBad)  // rare: the unit's first bad byte
                                    record_first_bad(sin, o, 16, lut, &err[win.w0 + k0],
                                                     uint64_t(rec.rel[k0]) + 16ull * (j0 + i));
                            } else {
                                const uint4 x = load16_shifted(sin, o, o & 3u);  // o mod 4 uniform
                                const uint4 ch = enc12(x, (fl0 >> 8) & 0xFFu, lut);
                                if (dd) *reinterpret_cast<uint4*>(d0 + 16 * i) = ch;
                                else *reinterpret_cast<uint4*>(sout + 16 * i) = ch;
                            }
                        }
                    };
                    // encode: a copy of the loop for each store target; decode: one
                    // copy with a uniform branch at its stores (smaller code measured
                    // faster there)
                    if constexpr (kDecode) whole(direct);
                    else if (direct) whole(std::true_type{});
                    else whole(std::false_type{});
                    if (!direct) run_len = RUN;
                    R = Rq;
                }
            }
            while (R < Rq) {
                // a mixed round: 32 V units (decode, V a lane) when the tile
                // has that many left, else up to 32 (one a lane)
                const uint32_t left = Rq - R;
                // wide only where every string of the window has aligned output
                const bool wide = kDecode && V > 1 && left >= 32u * V && win.dirm == 0xFFFFFFFFu;
                const uint32_t cnt = wide ? 32u * V : (left < 32u ? left : 32u);
                // the window's strings with units in [R, R + cnt)
                const bool has = win.un > 0 && win.us < R + cnt && win.us + win.un > R;
                if (kMixed && (__ballot_sync(0xffffffffu, has) & ~win.dirm) == 0) {
                    // ---- a mixed round: unit R + 32 v + lane for each v, of
                    //      whichever strings hold them (all stored from
                    //      registers). A lane finds each unit's string as the
                    //      last one starting at or below it: the strings that
                    //      start inside the round post their offset to one
                    //      32-bit mask a v and their index to a slot.
                    const int ks0 =
                        31 - __clz(__ballot_sync(0xffffffffu, win.un > 0 && win.us <= R));
                    const uint32_t d = win.us - R;
                    const bool starts = has && win.us > R;
                    __syncwarp();  // the previous round's slot reads are done
                    if (starts) rec.slot[d] = uint8_t(lane);
                    auto round = [&](auto vc) {
                        constexpr uint32_t NV = decltype(vc)::value;
                        uint32_t B[NV];
#pragma unroll
                        for (uint32_t v = 0; v < NV; ++v)
                            B[v] = __reduce_or_sync(
                                0xffffffffu, starts && (d >> 5) == v ? 1u << (d & 31u) : 0u);
                        __syncwarp();
                        const uint32_t le = 0xFFFFFFFFu >> (31 - lane);  // lanes <= this
                        int kv[NV];
                        int carry = ks0;  // the string of the last start below block v
#pragma unroll
                        for (uint32_t v = 0; v < NV; ++v) {
                            const uint32_t m = B[v] & le;
                            kv[v] = m ? int(rec.slot[32 * v + 31 - __clz(m)]) : carry;
                            if (v + 1 < NV && B[v])
                                carry = int(rec.slot[32 * v + 31 - __clz(B[v])]);
                        }
                        if constexpr (kDecode) {
                            // the NV units are decoded first and stored after, so
                            // their loads and table lookups overlap
                            uint3 outv[NV];
                            uint32_t nst[NV], eb[NV];
                            uint8_t* qv[NV];
#pragma unroll
                            for (uint32_t v = 0; v < NV; ++v) {
                                const uint32_t i = 32 * v + uint32_t(lane);
                                const int k = kv[v];
                                const uint32_t fl = rec.fl[k], us = rec.us[k];
                                const uint32_t j = R + i - us;
                                // an idle lane (i >= cnt) reads the buffer's
                                // start and stores nothing
                                const uint32_t o = i < cnt ? rec.lo[k] - p + delta + G * j : 0u;
                                const uint32_t nbl = fl & 0xFFu;
                                const bool part = j + 1 == rec.un[k] && nbl < G;
                                const uint32_t nb = part ? nbl : G;
                                qv[v] = dst + rec.dst[k] + int64_t(O) * j;
                                const uint4 c = load_unit16(sin, o);
                                uint32_t e0 = 0, e1 = 0, e2 = 0, e3 = 0;
                                const uint32_t lb = smem_addr(luts[(fl >> 8) & 0xFFu]);
                                outv[v] = pack4x24(decode4_at(c.x, lb, e0), decode4_at(c.y, lb, e1),
                                                   decode4_at(c.z, lb, e2), decode4_at(c.w, lb, e3));
                                // groups past a short unit's end are not the string's
                                eb[v] = e0 | (nb > 4 ? e1 : 0u) | (nb > 8 ? e2 : 0u) |
                                        (nb > 12 ? e3 : 0u);
                                nst[v] = i < cnt ? nb / 4 * 3 : 0u;  // a short unit: 3..9
                            }
#pragma unroll
                            for (uint32_t v = 0; v < NV; ++v) {
                                if (nst[v] == O) {
                                    uint32_t* ow = reinterpret_cast<uint32_t*>(qv[v]);
                                    ow[0] = outv[v].x;
                                    ow[1] = outv[v].y;
                                    ow[2] = outv[v].z;
                                } else if (nst[v]) {
                                    store_head_aligned(
                                        qv[v], make_uint4(outv[v].x, outv[v].y, outv[v].z, 0u),
                                        nst[v]);
                                }
                                if (nst[v] && (eb[v] & kBad)) {  // rare: the unit's first bad byte
                                    const int k = kv[v];
                                    const uint32_t fl = rec.fl[k];
                                    const uint32_t j = R + 32 * v + uint32_t(lane) - rec.us[k];
                                    record_first_bad(sin, rec.lo[k] - p + delta + G * j,
                                                     nst[v] / 3 * 4, luts[(fl >> 8) & 0xFFu],
                                                     &err[win.w0 + k],
                                                     uint64_t(rec.rel[k]) + 16ull * j);
                                }
                            }
                        } else if (uint32_t(lane) < cnt) {  // encode: one unit a lane
                            const int k = kv[0];
                            const uint32_t fl = rec.fl[k], us = rec.us[k];
                            const uint32_t j = R + uint32_t(lane) - us;
                            const uint32_t o = rec.lo[k] - p + delta + G * j;
                            const uint32_t nbl = fl & 0xFFu;
                            const bool part = j + 1 == rec.un[k] && nbl < G;
                            const uint8_t* lut = luts[(fl >> 8) & 0xFFu];
                            uint8_t* const qg = dst + rec.dst[k] + int64_t(O) * j;
                            const uint4 x = load16_shifted(sin, o, o & 3u);
                            if (part) {
                                uint32_t nout;
                                const uint4 ch = encode_last_unit(x, nbl, (fl & (1u << 16)) != 0,
                                                                  lut, &nout);
                                store_head_aligned(qg, ch, nout);
                            } else {
                                *reinterpret_cast<uint4*>(qg) = encode12(x.x, x.y, x.z, lut);
                            }
                        }
                    };
                    if (wide) round(std::integral_constant<uint32_t, V>{});
                    else round(std::integral_constant<uint32_t, 1>{});
                    R += cnt;
                    continue;
                }
                // ---- the units of one string in this tile (a piece), 32 a
                //      round with uniform addressing; the string's last unit,
                //      if shorter than G, is coded by its lane in the last round
                const int ks = 31 - __clz(__ballot_sync(0xffffffffu, win.un > 0 && win.us <= R));
                const uint32_t fl = rec.fl[ks], us = rec.us[ks], un = rec.un[ks];
                const uint32_t nbl = fl & 0xFFu;
                const bool padded = (fl & (1u << 16)) != 0;
                const uint32_t pend = Rq < us + un ? Rq : us + un;
                const uint8_t* lut = luts[(fl >> 8) & 0xFFu];
                const uint32_t olo = rec.lo[ks] - p + delta;  // sin offset of the string's unit 0
                uint8_t* const d_str = dst + rec.dst[ks];
                const bool direct = (reinterpret_cast<uintptr_t>(d_str) & (A - 1)) == 0;
                // output bytes of the string's last unit when it is shorter than G
                const uint32_t out_last =
                    kDecode ? nbl / 4 * 3
                            : nbl / 3 * 4 + (nbl % 3 == 0 ? 0u : padded ? 4u : nbl % 3 + 1);
                while (R < pend) {
                    const uint32_t cnt = pend - R < 32u ? pend - R : 32u;
                    const uint32_t j0 = R - us;
                    const bool ends = R + cnt == us + un && nbl < G;  // holds the short unit
                    if (!direct) run_at(d_str + int64_t(O) * j0, 32 * O);
                    // one unit a lane; kPart: the round holds the string's short
                    // last unit (in its last lane), a uniform choice
                    auto code_round = [&](auto part_round, auto direct_round) {
                        constexpr bool kPart = decltype(part_round)::value;
                        const bool direct = flag_value(direct_round);  // a constant in encode's copies
                        if (uint32_t(lane) >= cnt) return;
                        const uint32_t jj = j0 + lane;
                        const uint32_t o = olo + G * jj;
                        const bool part = kPart && uint32_t(lane) + 1 == cnt;
                        // global or run-buffer target: separate stores (uniform branch)
                        uint8_t* const qg = d_str + int64_t(O) * jj;
                        uint8_t* const qs = sout + run_len + O * lane;
                        if constexpr (kDecode) {
                            const uint4 c = load_unit16(sin, o);  // o mod 16 uniform
                            uint32_t e0 = 0, e1 = 0, e2 = 0, e3 = 0;
                            const uint32_t lb = smem_addr(lut);
                            const uint3 v =
                                pack4x24(decode4_at(c.x, lb, e0), decode4_at(c.y, lb, e1),
                                         decode4_at(c.z, lb, e2), decode4_at(c.w, lb, e3));
                            const uint32_t nbu = part ? nbl : 16u;
                            // groups past a short unit's end are not the string's
                            const uint32_t e = kPart ? e0 | (nbu > 4 ? e1 : 0u) |
                                                           (nbu > 8 ? e2 : 0u) | (nbu > 12 ? e3 : 0u)
                                                     : e0 | e1 | e2 | e3;
                            if (e & kBad)  // rare: the unit's first bad byte
                                record_first_bad(sin, o, nbu, lut, &err[win.w0 + ks],
                                                 uint64_t(rec.rel[ks]) + 16ull * jj);
                            if (kPart && direct && part) {
                                store_head_aligned(qg, make_uint4(v.x, v.y, v.z, 0u), out_last);
                            } else if (direct) {
                                uint32_t* ow = reinterpret_cast<uint32_t*>(qg);
                                ow[0] = v.x;
                                ow[1] = v.y;
                                ow[2] = v.z;
                            } else {
                                uint32_t* ow = reinterpret_cast<uint32_t*>(qs);
                                ow[0] = v.x;
                                ow[1] = v.y;
                                ow[2] = v.z;
                            }
                        } else {
                            const uint4 x = load16_shifted(sin, o, o & 3u);  // o mod 4 uniform
                            if (kPart && part) {
                                uint32_t nout;
                                const uint4 ch = encode_last_unit(x, nbl, padded, lut, &nout);
                                if (direct) store_head_aligned(qg, ch, nout);
                                else *reinterpret_cast<uint4*>(qs) = ch;
                            } else {
                                const uint4 ch = encode12(x.x, x.y, x.z, lut);
                                if (direct) *reinterpret_cast<uint4*>(qg) = ch;
                                else *reinterpret_cast<uint4*>(qs) = ch;
                            }
                        }
                    };
                    if constexpr (kDecode) {
                        if (ends) code_round(std::true_type{}, direct);
                        else code_round(std::false_type{}, direct);
                    } else if (direct) {
                        if (ends) code_round(std::true_type{}, std::true_type{});
                        else code_round(std::false_type{}, std::true_type{});
                    } else {
                        if (ends) code_round(std::true_type{}, std::false_type{});
                        else code_round(std::false_type{}, std::false_type{});
                    }
                    if (!direct) run_len += ends ? O * (cnt - 1) + out_last : O * cnt;
                    R += cnt;
                }
            }
            // more units below q can only be in later strings
            if (Rq < win.end_u || win.w0 + 32 >= n || win.next >= int64_t(q)) break;
            load_window<kDecode, G, A>(win, rec, win.w0 + 32, win.end_u, src_off, dst, dst_off,
                                       alph_id, tabs, n, P0, end, lane);
        }
    }
    if (run_len) flush();
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
        // always opted in: the static shared memory counts against the
        // default 48 KiB too
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

Occ g_enc_occ[4][64], g_dec_occ[4][64], g_encp_occ[4][64];
// Batches of up to this many alphabets may encode 8-unit tiles with pair
// tables when the caller asks (B64_TILE_PAIRS; two 8 KiB tables still leave
// room for two blocks an SM); 0 turns them off.
#ifndef B64_BATCH_ENC_PAIRS
#define B64_BATCH_ENC_PAIRS 2
#endif
constexpr int kPairAlphabets = B64_BATCH_ENC_PAIRS;

int unit_slot(int units) { return units == 1 ? 0 : units == 2 ? 1 : units == 4 ? 2 : 3; }

template <int U, bool kDecode, bool kPairs = false>
cudaError_t launch_tiles(const BatchArgs& a, const BatchTables& t, unsigned long long* err,
                         int blocks_per_sm, cudaStream_t st) {
    using Sh = TileShape<U, kDecode>;
    const DeviceInfo& di = device_info();
    cudaError_t e = cudaSuccess;
    // the pair tables' room is sized for kPairAlphabets, so the occupancy is one figure
    const size_t smem = Sh::kSmem + (kPairs ? size_t(kPairAlphabets) * 8192 : 0);
    Occ& slot = (kDecode ? g_dec_occ : kPairs ? g_encp_occ : g_enc_occ)[unit_slot(U)][di.device & 63];
    const int occ = occupancy(batch_tile_kernel<U, kDecode, kPairs>, Sh::kThreads, smem, smem,
                              slot, &e);
    if (e != cudaSuccess) return e;
    // blocks_per_sm (the tuner's second axis): fewer resident warps than fit
    const int bps = blocks_per_sm > 0 && blocks_per_sm < occ ? blocks_per_sm : occ;
    batch_tile_kernel<U, kDecode, kPairs><<<unsigned(di.sm_count * bps), Sh::kThreads, smem, st>>>(
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

// A string's output capacity: its encoded length, or 3 ceil(len / 4) for
// decode; rounded up to a multiple of 16 bytes with align16.
template <bool kDecode>
__device__ __forceinline__ int64_t capacity(const int64_t* __restrict__ src_off, int64_t i,
                                            const BatchTables& tabs,
                                            const uint8_t* __restrict__ alph_id, bool align16) {
    const uint64_t len = uint64_t(src_off[i + 1] - src_off[i]);
    uint64_t c;
    if (kDecode) {
        c = (len + 3) / 4 * 3;
    } else {
        const int al = alph_id ? (alph_id[i] & (kMaxAlphabets - 1)) : 0;
        c = enc_length(len, tabs.padded[al]);
    }
    return int64_t(align16 ? (c + 15) & ~uint64_t(15) : c);
}

template <bool kDecode>
__global__ void __launch_bounds__(kOffThreads)
    offsets_local_kernel(const int64_t* __restrict__ src_off, int64_t n,
                         const __grid_constant__ BatchTables tabs,
                         const uint8_t* __restrict__ alph_id, int64_t* __restrict__ dst_off,
                         bool align16) {
    __shared__ int64_t warp_sum[kOffThreads / 32];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t first = int64_t(blockIdx.x) * kOffItems;
    const int64_t i0 = first + int64_t(tid) * kScanItems;
    int64_t cap[kScanItems], sum = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        cap[j] = i0 + j < n ? capacity<kDecode>(src_off, i0 + j, tabs, alph_id, align16) : 0;
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

cudaError_t launch_batch(bool decode, const BatchArgs& a, const BatchTables& tabs, int tile,
                         void* workspace, cudaStream_t st) {
    const int units = tile & 0xFF, bps = (tile >> 8) & 0xFF;
    if (!decode) {
        encode_results_kernel<<<unsigned((a.n + 255) / 256), 256, 0, st>>>(a.src_off, a.n, tabs,
                                                                           a.alph_id, a.results);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        switch (units) {
            case 1: return launch_tiles<1, false>(a, tabs, nullptr, bps, st);
            case 2: return launch_tiles<2, false>(a, tabs, nullptr, bps, st);
            case 4: return launch_tiles<4, false>(a, tabs, nullptr, bps, st);
            default:
                if ((tile & B64_TILE_PAIRS) && tabs.n_alph >= 1 && tabs.n_alph <= kPairAlphabets)
                    return launch_tiles<8, false, true>(a, tabs, nullptr, bps, st);
                return launch_tiles<8, false>(a, tabs, nullptr, bps, st);
        }
    }
    unsigned long long* err = static_cast<unsigned long long*>(workspace);
    cudaError_t e = cudaMemsetAsync(err, 0xFF, size_t(a.n) * sizeof(uint64_t), st);  // kNoError
    if (e != cudaSuccess) return e;
    switch (units) {
        case 1: e = launch_tiles<1, true>(a, tabs, err, bps, st); break;
        case 2: e = launch_tiles<2, true>(a, tabs, err, bps, st); break;
        case 4: e = launch_tiles<4, true>(a, tabs, err, bps, st); break;
        default: e = launch_tiles<8, true>(a, tabs, err, bps, st); break;
    }
    if (e != cudaSuccess) return e;
    const unsigned grid = unsigned((a.n + 255) / 256);
    decode_batch_finalize_kernel<<<grid, 256, 0, st>>>(a.src, a.src_off, a.n, a.dst, a.dst_off,
                                                       tabs, a.alph_id, err, a.results);
    return cudaGetLastError();
}

}  // namespace b64

namespace b64 {

cudaError_t launch_batch_offsets(bool decode, bool align16, const int64_t* src_off, int64_t n,
                                 const BatchTables& tabs, const uint8_t* alph_id,
                                 int64_t* dst_off, cudaStream_t st) {
    const unsigned nblk = unsigned((n + kOffItems - 1) / kOffItems);
    if (nblk) {
        if (decode)
            offsets_local_kernel<true><<<nblk, kOffThreads, 0, st>>>(src_off, n, tabs, alph_id,
                                                                     dst_off, align16);
        else
            offsets_local_kernel<false><<<nblk, kOffThreads, 0, st>>>(src_off, n, tabs, alph_id,
                                                                      dst_off, align16);
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
