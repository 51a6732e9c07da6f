// MIME-style strict decode: CR, LF and space are skipped, everything else is
// decoded as by the single-buffer decoder (Sec. 2 and Sec. 3.2 of Mula &
// Lemire) on the characters that remain; error offsets are reported in the
// original input. The paper cites MIME only as motivation (Sec. 1); the
// whitespace removal and this single-pass design are this library's.
//
// One input: four kernels, no waits on other blocks:
//   1. count: every block takes 64 consecutive 4 KiB segments (rows of 32
//      lanes x 16 bytes; exact word-parallel tests for CR, LF and space),
//      counts each segment's data characters and last data byte, and writes
//      for each segment the prefix within its block, and the block's total;
//   2. scan (one block): block totals become block prefixes (plus the whole
//      input's count and last data byte), so a segment's global prefix is its
//      block's prefix plus its own: the index P of its first data character
//      and the last data byte before it (the group of four that straddles a
//      segment start is finished by the segment holding its second
//      character);
//   3. decode: every warp takes segments, each one's bulk (TMA) copy started
//      before the previous segment is worked on. Row by row it translates a
//      lane's 16 bytes through the table (6-bit value, bad = 0x80, whitespace
//      = 0xC0), counts the data characters from the class bits, scans the
//      counts over the warp and stores the values at their index with
//      predicated byte stores, in place (an index never exceeds its raw
//      position); it then decodes whole groups in place and writes exactly
//      the output bytes whose second character it holds, up to its first '='
//      or bad byte. Bad bytes and the first '=' are folded into status words
//      by atomic minima.
//   4. finalize (one thread): the padding and length rules on the compacted
//      stream, and the result.
// Inputs laid out as lines of L data characters (L a multiple of 4) and a
// fixed line break (CR LF or LF), detected from the first line, take a fast
// path in step 3: groups are decoded straight from the raw bytes at
// positions the layout gives, and a segment that does not fit the layout
// falls back to the general compaction. Many documents in one call (the
// batched entry point, further down) run the same steps with a memset of
// their status words, a per-document scan instead of the one-block scan, and
// a result per document.
// The only waits are on the decode kernels' own bulk copies, each bounded in
// time; one that runs out sets the timeout word, and the result becomes
// B64_E_TIMEOUT.
#include <mutex>
#include <type_traits>

#include "b64_internal.h"
#include "b64_smem.cuh"

// Line-layout fast path: whole groups four a lane for lines of 16 or more
// data characters (0: one group a lane for every line length).
#ifndef B64_MIME_UNITS
#define B64_MIME_UNITS 1
#endif

namespace b64 {
namespace {

constexpr int kWarps = 4;                               // warps per CTA, decode kernel
constexpr int kThreads = 32 * kWarps;
constexpr int kCountThreads = 256;                     // 8 warps
constexpr int kSegsPerBlock = 64;                       // segments per count block
constexpr int kScanThreads = 1024;
constexpr int kRows = 8;                                // rows of 32 lanes x 16 bytes
constexpr uint32_t kRow = 512;
constexpr uint32_t kSeg = kRow * kRows;                 // raw bytes per segment (4 KiB)
constexpr uint32_t kLead = 16;                          // buffer bytes before the segment
constexpr uint32_t kBuf = kLead + kSeg + 48;            // + room for shifted 16-byte reads
constexpr uint32_t kSpace = 0xC0u;                      // table class of CR, LF, space

// Segment state word: [flag:2][last data byte:8][data characters:54]. After
// the count kernel: flag 1 if the segment holds a data character, its last
// one, and its count. After the scan: the same fields for everything before
// the segment.
constexpr uint64_t kCountMask = (uint64_t(1) << 54) - 1;

// status[7] of the single-document call: the first segment whose whitespace
// does not sit where the line layout puts it (the one-pass kernel's check),
// or kNoSegment; the count, scan and decode kernels run only when it is set.
constexpr uint64_t kNoSegment = ~uint64_t(0);

__device__ uint32_t g_fault;

__host__ __device__ __forceinline__ uint64_t make_state(uint64_t flag, uint32_t last,
                                                        uint64_t count) {
    return (flag << 62) | (uint64_t(last & 0xFFu) << 54) | (count & kCountMask);
}
__host__ __device__ __forceinline__ uint64_t st_flag(uint64_t s) { return s >> 62; }
__host__ __device__ __forceinline__ uint32_t st_last(uint64_t s) {
    return uint32_t(s >> 54) & 0xFFu;
}
__host__ __device__ __forceinline__ uint64_t st_count(uint64_t s) { return s & kCountMask; }

// Four already-translated 6-bit values (one per byte, first in the low byte)
// -> their 24-bit value a<<18 | b<<12 | c<<6 | d. Each byte is masked to six
// bits first, so that a byte holding anything larger (a value past the end of
// the valid data: a raw byte or an earlier segment's value) cannot carry
// into the output bytes of the other values.
__device__ __forceinline__ uint32_t decode4_values(uint32_t w) {
    w &= 0x3F3F3F3Fu;
    const uint32_t a = w & 0xFFu, b = (w >> 8) & 0xFFu, c = (w >> 16) & 0xFFu, d = w >> 24;
    return ((a * 64u + b) * 64u + c) * 64u + d;
}

// Output bytes of the first j data characters.
__host__ __device__ __forceinline__ uint64_t bytes_for(uint64_t j) {
    const uint64_t r = j & 3;
    return 3 * (j >> 2) + (r ? r - 1 : 0);
}

// Bit 7 of each byte of x that equals the byte c (exact: no carries between bytes).
__device__ __forceinline__ uint32_t eq_bytes(uint32_t x, uint32_t c) {
    const uint32_t t = x ^ (c * 0x01010101u);
    return ~(((t & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | t) & 0x80808080u;
}
__device__ __forceinline__ uint32_t space_bytes(uint32_t x) {
    return eq_bytes(x, '\r') | eq_bytes(x, '\n') | eq_bytes(x, ' ');
}

__device__ __forceinline__ uint32_t byte_of(uint4 w, int k) {
    const uint32_t x = k < 4 ? w.x : k < 8 ? w.y : k < 12 ? w.z : w.w;
    return __byte_perm(x, 0, 0x4440u + (k & 3));
}

// Data characters of a 16-byte chunk (exact: every byte but CR, LF, space).
__device__ __forceinline__ uint32_t chunk_data(uint4 w) {
    return __popc(~space_bytes(w.x) & 0x80808080u) + __popc(~space_bytes(w.y) & 0x80808080u) +
           __popc(~space_bytes(w.z) & 0x80808080u) + __popc(~space_bytes(w.w) & 0x80808080u);
}

// The position + 1 (within the segment; off = the chunk's position) and value
// of a chunk's last data character, as (pos + 1) << 8 | byte; 0 if none.
__device__ __forceinline__ uint32_t chunk_last(uint4 w, uint32_t off) {
    const uint32_t d0 = ~space_bytes(w.x) & 0x80808080u, d1 = ~space_bytes(w.y) & 0x80808080u;
    const uint32_t d2 = ~space_bytes(w.z) & 0x80808080u, d3 = ~space_bytes(w.w) & 0x80808080u;
    // highest data byte: the top set bit of the four masks laid end to end
    const uint32_t hi = d3 ? 12 + (31 - __clz(d3)) / 8
                      : d2 ? 8 + (31 - __clz(d2)) / 8
                      : d1 ? 4 + (31 - __clz(d1)) / 8
                      : d0 ? (31 - __clz(d0)) / 8 : 0xFFu;
    return hi != 0xFFu ? ((off + hi + 1) << 8) | byte_of(w, int(hi)) : 0u;
}

// Data characters of a lane's kRows chunks (row r at kRow r + 16 lane), and
// the key of its last data character (chunk_last of the last chunk holding
// one). When every lane has data in its last row (the usual case), the key
// comes from that row alone; otherwise from each row that holds data, in
// order. Each row is used once, in order, so the rows need no longer life.
__device__ __forceinline__ uint32_t rows_count(const uint4 (&v)[kRows], int lane, uint32_t* key) {
    const uint32_t last = chunk_data(v[kRows - 1]);
    uint32_t count = last, k = 0;
    if (__all_sync(0xffffffffu, last != 0)) {
        k = chunk_last(v[kRows - 1], kRow * (kRows - 1) + 16 * lane);
#pragma unroll
        for (int r = 0; r < kRows - 1; ++r) count += chunk_data(v[r]);
    } else {
#pragma unroll
        for (int r = 0; r < kRows - 1; ++r) {
            const uint32_t c = chunk_data(v[r]);
            count += c;
            if (c) k = chunk_last(v[r], kRow * r + 16 * lane);
        }
        if (last) k = chunk_last(v[kRows - 1], kRow * (kRows - 1) + 16 * lane);
    }
    *key = k;
    return count;
}

// Segment bytes [0, len) in registers, row r of this lane in v[r]; bytes past
// len read as spaces.
__device__ __forceinline__ void load_rows(const uint8_t* seg_src, uint32_t len, bool aligned,
                                          int lane, uint4 (&v)[kRows]) {
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        const uint32_t off = kRow * r + 16 * lane;
        if (aligned && off + 16 <= len) {
            v[r] = *reinterpret_cast<const uint4*>(seg_src + off);
        } else {
            uint8_t* b = reinterpret_cast<uint8_t*>(&v[r]);
            for (int k = 0; k < 16; ++k) b[k] = off + k < len ? seg_src[off + k] : uint8_t(' ');
        }
    }
}

__device__ __forceinline__ uint32_t warp_scan_add32(uint32_t v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}
__device__ __forceinline__ uint32_t warp_scan_max32(uint32_t v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o && u > v) v = u;
    }
    return v;
}

// ---------------------------------------------------------------- 1. count
// Block b: segments [64 b, 64 b + 64). states[s] = (data characters and last
// data byte of the segments before s in its block); totals[b] = the block's.
__global__ void __launch_bounds__(kCountThreads, 4)
    mime_count_kernel(const uint8_t* __restrict__ src, uint64_t m,
                      unsigned long long* __restrict__ states,
                      unsigned long long* __restrict__ totals, uint64_t nseg,
                      const unsigned long long* __restrict__ status) {
    __shared__ uint32_t s_cnt[kSegsPerBlock], s_key[kSegsPerBlock];
    wait_prior_grid();  // the one-pass kernel's status words
    if (status[7] == kNoSegment) return;  // the one-pass kernel decoded everything
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool aligned = (reinterpret_cast<uintptr_t>(src) & 15u) == 0;
    const uint64_t first = uint64_t(blockIdx.x) * kSegsPerBlock;
    for (int j = warp; j < kSegsPerBlock; j += kCountThreads / 32) {
        const uint64_t seg = first + j;
        uint32_t count = 0, key = 0;
        if (seg < nseg) {
            const uint64_t base = seg * kSeg;
            const uint32_t len = uint32_t(m - base < kSeg ? m - base : kSeg);
            uint4 v[kRows];
            load_rows(src + base, len, aligned, lane, v);
            count = __reduce_add_sync(0xffffffffu, rows_count(v, lane, &key));
            key = __reduce_max_sync(0xffffffffu, key);
        }
        if (lane == 0) {
            s_cnt[j] = count;
            s_key[j] = key ? (uint32_t(j + 1) << 8) | (key & 0xFFu) : 0u;  // block-local order
        }
    }
    __syncthreads();
    if (warp == 0) {  // two segments per lane
        const uint32_t c0 = s_cnt[2 * lane], c1 = s_cnt[2 * lane + 1];
        const uint32_t k0 = s_key[2 * lane], k1 = s_key[2 * lane + 1];
        const uint32_t incl = warp_scan_add32(c0 + c1, lane);
        const uint32_t kincl = warp_scan_max32(k0 > k1 ? k0 : k1, lane);
        uint32_t kex = __shfl_up_sync(0xffffffffu, kincl, 1);
        if (lane == 0) kex = 0;
        const uint32_t ex = incl - c0 - c1;
        const uint64_t s0 = first + 2 * lane;
        if (s0 < nseg) states[s0] = make_state(kex != 0, kex & 0xFFu, ex);
        const uint32_t kmid = k0 > kex ? k0 : kex;
        if (s0 + 1 < nseg) states[s0 + 1] = make_state(kmid != 0, kmid & 0xFFu, ex + c0);
        if (lane == 31) totals[blockIdx.x] = make_state(kincl != 0, kincl & 0xFFu, incl);
    }
}

// The layout word of an input whose first whitespace byte is at f (f = the
// input's first 1024 bytes if none): L = f if f is a multiple of 4
// (at least 4) and the bytes at f are CR LF or a lone LF.
__device__ __forceinline__ uint32_t line_layout_word(const uint8_t* p, uint64_t len, uint32_t f) {
    if (f >= 1024 || f < 4 || f % 4 != 0 || uint64_t(f) >= len) return 0;
    if (p[f] == '\n') return f | (1u << 16);
    if (p[f] == '\r' && uint64_t(f) + 1 < len && p[f + 1] == '\n') return f | (2u << 16);
    return 0;
}

// ---------------------------------------------------------------- 2. scan
// One block: totals[b] = (data characters before block b, last data byte
// before it); status[5] = the whole input's (count, last data byte).
constexpr int kScanItems = 8;

__global__ void __launch_bounds__(kScanThreads)
    mime_scan_kernel(unsigned long long* __restrict__ totals, uint64_t nblk,
                     unsigned long long* __restrict__ status, const uint8_t* __restrict__ src,
                     uint64_t m) {
    __shared__ uint64_t warp_sum[kScanThreads / 32];
    __shared__ uint64_t warp_key[kScanThreads / 32];
    __shared__ uint32_t first_space;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    wait_prior_grid();  // the count kernel's totals and the status words
    if (status[7] == kNoSegment) return;  // the one-pass kernel decoded everything
    // the decode kernel recomputes the error and '=' words: what the one-pass
    // kernel left there came from counts that may be wrong past status[7]
    if (tid < 3) status[tid] = kNoError;
    // status[6] = the line layout word if the input starts with a line of L
    // data characters and CR LF or LF, L a multiple of 4 below 1024 (the
    // decode kernel's fast path, checked there segment by segment), else 0
    if (tid == 0) first_space = kScanThreads;
    __syncthreads();
    if (uint64_t(tid) < m) {
        const uint32_t c = src[tid];
        if (c == '\r' || c == '\n' || c == ' ') atomicMin(&first_space, uint32_t(tid));
    }
    __syncthreads();
    if (tid == 0) status[6] = line_layout_word(src, m, first_space);
    uint64_t carry = 0, carry_key = 0;  // key: (block + 1) << 8 | last byte, 0 = none
    for (uint64_t base = 0; base < nblk; base += uint64_t(kScanThreads) * kScanItems) {
        const uint64_t i0 = base + uint64_t(tid) * kScanItems;
        uint64_t cnt[kScanItems], keys[kScanItems];
        uint64_t sum = 0, kmax = 0;
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            const uint64_t i = i0 + j;
            const uint64_t st = i < nblk ? totals[i] : 0;
            cnt[j] = st_count(st);
            keys[j] = st_flag(st) ? ((i + 1) << 8) | st_last(st) : 0;
            sum += cnt[j];
            kmax = keys[j] > kmax ? keys[j] : kmax;
        }
        uint64_t incl = sum, ikey = kmax;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t u = __shfl_up_sync(0xffffffffu, incl, o);
            const uint64_t uk = __shfl_up_sync(0xffffffffu, ikey, o);
            if (lane >= o) {
                incl += u;
                ikey = uk > ikey ? uk : ikey;
            }
        }
        if (lane == 31) {
            warp_sum[warp] = incl;
            warp_key[warp] = ikey;
        }
        __syncthreads();
        if (warp == 0) {
            uint64_t x = warp_sum[lane], xk = warp_key[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t u = __shfl_up_sync(0xffffffffu, x, o);
                const uint64_t uk = __shfl_up_sync(0xffffffffu, xk, o);
                if (lane >= o) {
                    x += u;
                    xk = uk > xk ? uk : xk;
                }
            }
            warp_sum[lane] = x;
            warp_key[lane] = xk;
        }
        __syncthreads();
        uint64_t run = carry + (warp ? warp_sum[warp - 1] : 0) + incl - sum;
        // keys before this thread's items: carried, earlier warps, earlier lanes
        uint64_t rkey = carry_key;
        if (warp && warp_key[warp - 1] > rkey) rkey = warp_key[warp - 1];
        const uint64_t lane_prev = __shfl_up_sync(0xffffffffu, ikey, 1);
        if (lane && lane_prev > rkey) rkey = lane_prev;
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            if (i0 + j < nblk) totals[i0 + j] = make_state(rkey != 0, uint32_t(rkey & 0xFFu), run);
            run += cnt[j];
            rkey = keys[j] > rkey ? keys[j] : rkey;
        }
        carry += warp_sum[kScanThreads / 32 - 1];
        if (warp_key[kScanThreads / 32 - 1] > carry_key) carry_key = warp_key[kScanThreads / 32 - 1];
        __syncthreads();  // warp_sum / warp_key are rewritten by the next chunk
    }
    if (tid == 0) status[5] = make_state(carry_key != 0, uint32_t(carry_key & 0xFFu), carry);
}

// ---------------------------------------------------------------- 3. decode
// Bounded wait on a bulk copy's barrier: false after limit_ns.
__device__ __forceinline__ bool wait_copy(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (;;) {
        for (int i = 0; i < 16; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_timer_ns() - t0 > limit_ns) return false;
    }
}

// One staged segment (its bytes at buf[kLead ..], the tail past the document's
// end reading as spaces), decoded by one warp: the row-by-row compaction of
// the 6-bit values, the status words (first bad byte and first '=', offsets
// relative to raw_base / the document), the whole groups and the output bytes
// whose second character the segment holds. P: data characters before the
// segment in its document; prev_last: the last data byte before it.
__device__ __forceinline__ void copy_out(const uint8_t* buf, uint32_t skip, uint32_t nout,
                                         uint8_t* __restrict__ q, int lane);

__device__ __forceinline__ void decode_segment(uint8_t* buf, const uint8_t* lut, int flags,
                                               int lane, uint64_t P, uint32_t prev_last,
                                               uint64_t raw_base, uint8_t* __restrict__ out_doc,
                                               unsigned long long* st3) {
    const uint64_t base = raw_base;
    // ---- row by row (512 bytes = four sub-rows of 128; lane L takes word L
    //      of each): translate, count, scan, and store each value at
    //      buf[kLead + s + index], s = P mod 4, so that whole groups of four
    //      start on 16-byte boundaries. A value's position never passes its
    //      raw byte by more than 3, so the next row is read before any lane
    //      writes (the only raw bytes a row's stores can reach).
    const uint32_t s = uint32_t(P & 3);
    const uint32_t* raw32 = reinterpret_cast<const uint32_t*>(buf + kLead);
    uint32_t bad_raw = 0xFFFFFFFFu, eq_raw = 0xFFFFFFFFu, eq_comp = 0xFFFFFFFFu,
             stop = 0xFFFFFFFFu;
    uint32_t rowbase = 0;
    uint32_t xr[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) xr[j] = raw32[32 * j + lane];
#pragma unroll 1
    for (int r = 0; r < kRows; ++r) {
        uint32_t xn[4] = {0u, 0u, 0u, 0u};
        if (r + 1 < kRows) {
#pragma unroll
            for (int j = 0; j < 4; ++j) xn[j] = raw32[128 * (r + 1) + 32 * j + lane];
        }
        uint32_t T[4], dm[4], badm[4], C = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t x = xr[j];
            const uint32_t t0 = lut[x & 0xFFu], t1 = lut[(x >> 8) & 0xFFu];
            const uint32_t t2 = lut[(x >> 16) & 0xFFu], t3 = lut[x >> 24];
            T[j] = t0 | (t1 << 8) | (t2 << 16) | (t3 << 24);
            const uint32_t b7 = T[j] & 0x80808080u, b6 = (T[j] << 1) & 0x80808080u;
            dm[j] = ~(b7 & b6) & 0x80808080u;  // not whitespace (0xC0)
            badm[j] = b7 & ~b6;                // bad or '=' (0x80)
            C |= uint32_t(__popc(dm[j])) << (8 * j);
        }
        // four 8-bit counts scanned at once (a sub-row holds at most 128)
        const uint32_t incl = warp_scan_add32(C, lane);
        const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
        const uint32_t ex = incl - C;
        __syncwarp();  // row r and row r + 1 are read everywhere before any lane writes
        uint32_t base = rowbase;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t idx = base + ((ex >> (8 * j)) & 0xFFu);
            uint8_t* out = buf + kLead + s + idx;
            uint32_t q = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const uint32_t v = (T[j] >> (8 * i)) & 0xFFu;
                if (v < kSpace) {
                    out[q] = uint8_t(v);
                    ++q;
                }
            }
            if (badm[j]) {  // rare: the word's first bad byte and first '='
                uint32_t qq = 0;
                for (int i = 0; i < 4; ++i) {
                    const uint32_t v = (T[j] >> (8 * i)) & 0xFFu;
                    if (v == kSpace) continue;
                    if (v & kBad) {
                        const uint32_t ch = (xr[j] >> (8 * i)) & 0xFFu;
                        const uint32_t rawpos = kRow * r + 128 * j + 4 * lane + i;
                        if (stop == 0xFFFFFFFFu || idx + qq < stop) stop = idx + qq;
                        if (ch == '=' && (flags & 1)) {
                            if (eq_raw == 0xFFFFFFFFu || rawpos < eq_raw) {
                                eq_raw = rawpos;
                                eq_comp = idx + qq;
                            }
                        } else if (bad_raw == 0xFFFFFFFFu || rawpos < bad_raw) {
                            bad_raw = rawpos;
                        }
                        break;
                    }
                    ++qq;
                }
            }
            base += (tot >> (8 * j)) & 0xFFu;
        }
        rowbase = base;
#pragma unroll
        for (int j = 0; j < 4; ++j) xr[j] = xn[j];
    }
    const uint32_t count = rowbase;
    stop = __reduce_min_sync(0xffffffffu, stop);
    if (stop != 0xFFFFFFFFu) {
        bad_raw = __reduce_min_sync(0xffffffffu, bad_raw);
        eq_raw = __reduce_min_sync(0xffffffffu, eq_raw);
        eq_comp = __reduce_min_sync(0xffffffffu, eq_comp);
        if (lane == 0) {
            if (bad_raw != 0xFFFFFFFFu) atomicMin(st3 + 0, base + bad_raw);
            if (eq_raw != 0xFFFFFFFFu) {
                atomicMin(st3 + 1, base + eq_raw);
                atomicMin(st3 + 2, P + eq_comp);
            }
        }
    }

    // ---- whole groups in place: 16 values -> 12 bytes. The value of data
    //      character P + i sits at buf[kLead + s + i], so the group holding P
    //      starts at buf[kLead] and group g at buf[kLead + 16 g]; the value
    //      before P goes to buf[kLead + s - 1]
    if (lane == 0 && s) buf[kLead + s - 1] = lut[prev_last];
    __syncwarp();
    const uint32_t jend = stop < count ? stop : count;
    const uint64_t ob = bytes_for(P), oe = bytes_for(P + jend);
    const uint32_t nout = uint32_t(oe > ob ? oe - ob : 0);
    const uint32_t skip = s ? s - 1 : 0;  // bytes of the first group written before P
    const uint32_t ngroups = (s + jend + 15) / 16;
#pragma unroll 1
    for (uint32_t g0 = 0; g0 < ngroups; g0 += 32) {
        const uint32_t g = g0 + lane;
        uint3 o = make_uint3(0, 0, 0);
        if (g < ngroups) {
            const uint4 c = *reinterpret_cast<const uint4*>(buf + kLead + 16 * g);
            o = pack4x24(decode4_values(c.x), decode4_values(c.y), decode4_values(c.z),
                         decode4_values(c.w));
        }
        __syncwarp();  // this round's values are read before any lane overwrites them
        if (g < ngroups) {
            uint32_t* ow = reinterpret_cast<uint32_t*>(buf + 12 * g);
            ow[0] = o.x;
            ow[1] = o.y;
            ow[2] = o.z;
        }
    }
    __syncwarp();
    copy_out(buf, skip, nout, out_doc + ob, lane);
}

// Copies buf[skip .. skip + nout) to global q: 16-byte stores at aligned
// addresses, each built from two aligned 16-byte shared loads; bytes at the
// edges. Reads up to 32 bytes past skip + nout. Warp-collective. The word
// offset of the source within its 16 bytes is the same for every store, so
// the loop has one copy per offset with the words picked at compile time.
template <uint32_t SW>
__device__ __forceinline__ void copy_out_body(const uint8_t* buf, uint32_t A0, uint32_t n16,
                                              uint32_t sb, uint8_t* __restrict__ q, int lane) {
    for (uint32_t i = lane; i < n16; i += 32) {
        const uint32_t A = A0 + 16 * i;
        const uint4 a = *reinterpret_cast<const uint4*>(buf + A);
        const uint4 b = *reinterpret_cast<const uint4*>(buf + A + 16);
        const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        *reinterpret_cast<uint4*>(q + 16 * i) =
            make_uint4(__funnelshift_r(w[SW], w[SW + 1], sb), __funnelshift_r(w[SW + 1], w[SW + 2], sb),
                       __funnelshift_r(w[SW + 2], w[SW + 3], sb),
                       __funnelshift_r(w[SW + 3], w[SW + 4], sb));
    }
}
__device__ __forceinline__ void copy_out(const uint8_t* buf, uint32_t skip, uint32_t nout,
                                         uint8_t* __restrict__ q, int lane) {
    const uint32_t head = uint32_t((16 - (reinterpret_cast<uintptr_t>(q) & 15)) & 15);
    const uint32_t h = head < nout ? head : nout;
    if (lane < int(h)) q[lane] = buf[skip + lane];
    const uint32_t body = (nout - h) & ~15u;
    const uint32_t o0 = skip + h, sw = (o0 & 15) >> 2, sb = 8 * (o0 & 3);
    const uint32_t A0 = o0 & ~15u;
    switch (sw) {  // the same in every lane
        case 0: copy_out_body<0>(buf, A0, body / 16, sb, q + h, lane); break;
        case 1: copy_out_body<1>(buf, A0, body / 16, sb, q + h, lane); break;
        case 2: copy_out_body<2>(buf, A0, body / 16, sb, q + h, lane); break;
        default: copy_out_body<3>(buf, A0, body / 16, sb, q + h, lane); break;
    }
    for (uint32_t i = h + body + lane; i < nout; i += 32) q[i] = buf[skip + i];
}

// Fast path for a whole segment of a document laid out as lines of exactly
// L data characters, each followed by a line break of e bytes (CR LF, e = 2,
// or a lone LF, e = 1), with L a multiple of 4 (76 for MIME, 64 for PEM): no
// group of four then straddles a line break, and data character j sits at
// raw position (L + e) floor(j / L) + j mod L. The warp
// decodes the groups straight from the raw bytes (four translations, one
// 24-bit value and three output bytes a group), writing the output in place
// below the bytes still to be read, and checks on the way that the segment
// really has that layout: every byte it takes as data is in the alphabet
// (not '=', not whitespace) and every byte it skips is whitespace. Only then
// does it copy the output out (kLinesDone). If the count of data characters
// before the segment does not fit the layout it returns kLinesNo at once,
// the staged bytes untouched; if a check fails it returns kLinesSpoilt
// (whitespace sits where the layout has it, but some data byte is outside the
// alphabet or is '=') or kLinesIrregular (a whitespace byte where the layout
// has data, or a break position holding something else): nothing has been
// written to global memory, but the staged bytes are spoilt and the caller
// stages the segment again for the general path (which also finds the
// segment's errors). S: the segment's raw start in the document; P: the data
// characters before it; prev_last: the last data byte before it; delta: the
// segment's first byte sits at buf + kLead + delta (0 to 15; nonzero only for
// L >= 16, and even for CR LF breaks, so that a unit's three 8-byte loads
// still hold its bytes and the break's).
enum LinesResult { kLinesNo, kLinesDone, kLinesSpoilt, kLinesIrregular };

// The line layout's constants (L = 0: the input does not start with it).
// word: L | eol << 16 (eol = 2 for CR LF, 1 for LF), 0 for none.
struct LineLayout {
    uint32_t L = 0, eol = 0, Q = 0;  // data characters a line; break bytes; raw bytes a line
    uint32_t inv = 0;                // 2^32 / L rounded up: t / L = umulhi(t, inv) for t < 2^13
    uint32_t seg_q = 0, seg_r = 0;   // kSeg = seg_q Q + seg_r
    __device__ explicit LineLayout(uint32_t word) {
        if (word) {
            L = word & 0xFFFFu;
            eol = word >> 16;
            Q = L + eol;
            inv = 0xFFFFFFFFu / L + 1u;
            seg_q = kSeg / Q;
            seg_r = kSeg - seg_q * Q;
        }
    }
};


// S = k Q + r is the segment's raw start in the document; kCrLf: breaks
// are CR LF (ly.eol == 2), so every group starts at an even raw offset.
template <bool kCrLf>
__device__ LinesResult decode_lines(uint8_t* buf, const uint8_t* lut, int lane,
                                    const LineLayout& ly, uint64_t k, uint32_t r, uint64_t P,
                                    uint32_t prev_last, uint8_t* __restrict__ out_doc,
                                    uint32_t delta) {
    const uint32_t L = ly.L, Q = ly.Q, eol = kCrLf ? 2u : 1u;
    if (delta && (L < 16 || (kCrLf && (delta & 1u)))) return kLinesNo;  // not for this path
    // data characters before S, and before the segment's end, in the layout
    if (k * L + (r < L ? r : L) != P) return kLinesNo;  // it does not hold up to here
    uint64_t k1 = k + ly.seg_q;
    uint32_t r1 = r + ly.seg_r;
    if (r1 >= Q) {
        r1 -= Q;
        ++k1;
    }
    const uint64_t P1 = k1 * L + (r1 < L ? r1 : L);
    const uint8_t* raw = buf + kLead;
    // raw offset from buf + kLead of data character P + d (d < 4096 + L): the
    // column of P in its line, and the raw offset of that line's start
    const uint32_t rP = r < L ? r : 0;
    const int32_t off0 = (r < L ? -int32_t(r) : int32_t(Q - r)) + int32_t(delta);
    auto raw_of = [&](uint32_t d) -> uint32_t {
        const uint32_t t = rP + d, line = __umulhi(t, ly.inv);
        return uint32_t(off0) + line * eol + t;  // line Q + (t - line L)
    };
    // bad: bit 7 of every data value OR-ed (outside the alphabet, '=' or
    // whitespace), bit 6 also for whitespace (kSpace); viol: a layout violation
    uint32_t bad = 0, viol = 0;
    // the skipped bytes: break j at raw offsets L - r + j Q (and one more
    // for CR LF)
    const uint8_t* seg = raw + delta;
    for (int32_t rel = int32_t(L) - int32_t(r) + lane * int32_t(Q); rel < int32_t(kSeg);
         rel += 32 * int32_t(Q)) {
        if (rel >= 0 && lut[seg[rel]] != kSpace) viol = 1u;
        if (kCrLf && rel + 1 >= 0 && rel + 1 < int32_t(kSeg) && lut[seg[rel + 1]] != kSpace)
            viol = 1u;
    }
    // groups: the one holding P (edge A: it started before the segment), the
    // whole ones, the one holding P1 - 1 (edge B: it ends after the segment)
    const uint32_t rA = uint32_t(P & 3), rB = uint32_t(P1 & 3);
    const uint32_t cA = rA ? 4 - rA : 0;              // edge A's output bytes; first whole d
    const uint32_t nfull = uint32_t((P1 - P - cA) / 4);
    const uint32_t base = kLead;                      // whole group i at buf[base + 3 i]
    // edge values, one a lane: lanes 0..3 value t of group A (t = rA - 1 is
    // the data byte before the segment), lanes 4..7 value t - 4 of group B
    uint32_t ea = 0, eb = 0;
    if (lane < 4 && rA && uint32_t(lane) + 1 >= rA) {
        const uint32_t t = uint32_t(lane);
        const uint32_t v = t + 1 == rA ? lut[prev_last] : lut[raw[raw_of(t - rA)]];
        if (t + 1 != rA) bad |= v & 0xC0u;
        ea = (v & 63u) << (6 * (3 - t));
    } else if (lane >= 4 && lane < 8 && rB >= 2 && uint32_t(lane) - 4 < rB) {
        const uint32_t t = uint32_t(lane) - 4;
        const uint32_t v = lut[raw[raw_of(cA + 4 * nfull + t)]];
        bad |= v & 0xC0u;
        eb = (v & 63u) << (6 * (3 - t));
    }
    const uint32_t wA = __reduce_or_sync(0xffffffffu, ea);
    const uint32_t wB = __reduce_or_sync(0xffffffffu, eb);
    if (B64_MIME_UNITS && L >= 16) {
        // whole groups four a lane: unit i holds the 16 data characters from
        // cA + 16 i (the last unit possibly fewer groups). A unit starts at a
        // column that is a multiple of 4, and L >= 16 is one too, so it
        // crosses at most one line break, between two of its words: the words
        // before the break are the 16 raw bytes at the unit's start, the rest
        // the same bytes eol further on. Units go 32 a round; every read of a
        // round comes before its writes (unit i's 12 output bytes at
        // buf[base + 12 i]), and a round's writes (below base + 384 (r + 1))
        // stay below the next round's reads (unit i's raw offset is at least
        // 16 i, its first 8-byte load at most 7 below it).
        const uint32_t nunits = (nfull + 3) / 4;
        const uint32_t lb = smem_addr(lut);
        auto unit_round = [&](uint32_t u0, auto checked) {
            constexpr bool kChecked = decltype(checked)::value;
            const uint32_t i = u0 + uint32_t(lane);
            uint32_t ng = 4;  // groups of the lane's unit
            if constexpr (kChecked) ng = i < nunits ? (nfull - 4 * i < 4 ? nfull - 4 * i : 4u) : 0u;
            uint3 v = make_uint3(0u, 0u, 0u);
            if (!kChecked || ng) {
                const uint32_t t = rP + cA + 16 * i, line = __umulhi(t, ly.inv);
                const uint32_t col = t - line * L;                    // a multiple of 4
                const uint32_t ro = uint32_t(off0) + line * eol + t;  // raw_of(cA + 16 i)
                const uint32_t A = ro & ~7u, sh = ro & 7u;
                const uint2 x0 = *reinterpret_cast<const uint2*>(raw + A);
                const uint2 x1 = *reinterpret_cast<const uint2*>(raw + A + 8);
                const uint2 x2 = *reinterpret_cast<const uint2*>(raw + A + 16);
                // W0..W3: raw bytes sh .. sh + 15; W4: the low bytes of sh + 16 ..
                const bool o1 = sh >= 4;
                const uint32_t sb = 8 * (sh & 3u);
                const uint32_t a0 = o1 ? x0.y : x0.x, a1 = o1 ? x1.x : x0.y,
                               a2 = o1 ? x1.y : x1.x, a3 = o1 ? x2.x : x1.y,
                               a4 = o1 ? x2.y : x2.x;
                const uint32_t w0 = __funnelshift_r(a0, a1, sb), w1 = __funnelshift_r(a1, a2, sb);
                const uint32_t w2 = __funnelshift_r(a2, a3, sb), w3 = __funnelshift_r(a3, a4, sb);
                const uint32_t w4 = a4 >> sb;  // its eol low bytes are loaded (sh + eol <= 8)
                // past the break (after tb = L - col >= 4 data characters) the
                // words are the same bytes eol further on
                const uint32_t tb = L - col;
                const uint32_t c1 = tb <= 4 ? __funnelshift_r(w1, w2, 8 * eol) : w1;
                const uint32_t c2 = tb <= 8 ? __funnelshift_r(w2, w3, 8 * eol) : w2;
                const uint32_t c3 = tb <= 12 ? __funnelshift_r(w3, w4, 8 * eol) : w3;
                uint32_t e0 = 0, e1 = 0, e2 = 0, e3 = 0;
                v = pack4x24(decode4_at(w0, lb, e0), decode4_at(c1, lb, e1),
                             decode4_at(c2, lb, e2), decode4_at(c3, lb, e3));
                if constexpr (kChecked)
                    bad |= e0 | (ng > 1 ? e1 : 0u) | (ng > 2 ? e2 : 0u) | (ng > 3 ? e3 : 0u);
                else
                    bad |= e0 | e1 | e2 | e3;
            }
            __syncwarp();
            if constexpr (kChecked) {
                if (ng) store_head_aligned(buf + base + 12 * i, make_uint4(v.x, v.y, v.z, 0u), 3 * ng);
            } else {
                uint32_t* ow = reinterpret_cast<uint32_t*>(buf + base + 12 * i);
                ow[0] = v.x;
                ow[1] = v.y;
                ow[2] = v.z;
            }
            __syncwarp();
        };
        const uint32_t nwu = nfull / 128 * 32;  // units of the rounds of 32 whole units
        for (uint32_t u0 = 0; u0 < nwu; u0 += 32) unit_round(u0, std::false_type{});
        if (nwu < nunits) unit_round(nwu, std::true_type{});
    } else {
        // whole groups, 128 a round: every read of a round comes before its
        // writes, and a round's writes (below 384 (r + 1)) stay below the next
        // round's reads (a group's raw offset is at least 4 times its index)
        constexpr int kPer = 4;  // groups a lane per round, 32 apart
        auto round = [&](uint32_t i0, auto checked) {
            uint32_t q[kPer];
#pragma unroll
            for (int u = 0; u < kPer; ++u) {
                const uint32_t i = i0 + 32 * u + lane;
                q[u] = 0;
                if (!decltype(checked)::value || i < nfull) {
                    const uint32_t ro = raw_of(cA + 4 * i);
                    uint32_t x;
                    if constexpr (kCrLf) {  // even offsets: two 16-bit loads
                        x = __byte_perm(*reinterpret_cast<const uint16_t*>(raw + ro),
                                        *reinterpret_cast<const uint16_t*>(raw + ro + 2), 0x5410u);
                    } else {  // any offset: two aligned words, one shift
                        const uint32_t* w = reinterpret_cast<const uint32_t*>(raw + (ro & ~3u));
                        x = __funnelshift_r(w[0], w[1], 8 * (ro & 3u));
                    }
                    const uint32_t a = lut[x & 0xFFu], b = lut[(x >> 8) & 0xFFu];
                    const uint32_t c = lut[(x >> 16) & 0xFFu], d = lut[x >> 24];
                    bad |= a | b | c | d;
                    q[u] = ((a * 64u + b) * 64u + c) * 64u + d;
                }
            }
            __syncwarp();
#pragma unroll
            for (int u = 0; u < kPer; ++u) {
                const uint32_t i = i0 + 32 * u + lane;
                if (!decltype(checked)::value || i < nfull) {
                    uint8_t* o = buf + base + 3 * i;
                    o[0] = uint8_t(q[u] >> 16);
                    o[1] = uint8_t(q[u] >> 8);
                    o[2] = uint8_t(q[u]);
                }
            }
            __syncwarp();
        };
        const uint32_t nwhole = nfull / (32 * kPer) * (32 * kPer);
        for (uint32_t i0 = 0; i0 < nwhole; i0 += 32 * kPer) round(i0, std::false_type{});
        if (nwhole < nfull) round(nwhole, std::true_type{});
    }
    if (__any_sync(0xffffffffu, viol != 0 || (bad & 0x40u) != 0)) return kLinesIrregular;
    if (__any_sync(0xffffffffu, bad & 0x80u)) return kLinesSpoilt;
    if (uint32_t(lane) < cA)  // bytes rA - 1 .. 2 of edge A
        buf[base - cA + lane] = uint8_t(wA >> (16 - 8 * (rA - 1 + lane)));
    if (rB >= 2 && uint32_t(lane) + 1 < rB)  // bytes 0 .. rB - 2 of edge B
        buf[base + 3 * nfull + lane] = uint8_t(wB >> (16 - 8 * lane));
    __syncwarp();
    const uint64_t ob = bytes_for(P);
    copy_out(buf, base - cA, uint32_t(bytes_for(P1) - ob), out_doc + ob, lane);
    return kLinesDone;
}

__device__ __forceinline__ LinesResult decode_segment_lines(uint8_t* buf, const uint8_t* lut,
                                                            int lane, const LineLayout& ly,
                                                            uint64_t k, uint32_t r, uint64_t P,
                                                            uint32_t prev_last,
                                                            uint8_t* __restrict__ out_doc,
                                                            uint32_t delta = 0) {
    return ly.eol == 2
               ? decode_lines<true>(buf, lut, lane, ly, k, r, P, prev_last, out_doc, delta)
               : decode_lines<false>(buf, lut, lane, ly, k, r, P, prev_last, out_doc, delta);
}

__global__ void __launch_bounds__(kThreads, 6)
    mime_decode_kernel(const uint8_t* __restrict__ src, uint64_t m, uint8_t* __restrict__ dst,
                       const __grid_constant__ DecodeTable tab, int flags,
                       unsigned long long* __restrict__ status,
                       const unsigned long long* __restrict__ states,
                       const unsigned long long* __restrict__ totals, uint64_t nseg,
                       uint64_t wait_limit_ns) {
    __shared__ __align__(256) uint8_t lut[256];  // 0..63, 0x80 (bad or '='), kSpace
    __shared__ __align__(16) uint8_t bufs[kWarps][2][kBuf];
    __shared__ uint64_t bars[kWarps][2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < 64; i += kThreads) reinterpret_cast<uint32_t*>(lut)[i] = tab.w[i];
    __syncthreads();
    if (tid == 0) lut['\r'] = lut['\n'] = lut[' '] = uint8_t(kSpace);
    if (lane == 0) {
        mbar_init(&bars[warp][0], 1);
        mbar_init(&bars[warp][1], 1);
        fence_mbar_init();
    }
    __syncthreads();  // the only block-wide barrier: tables and barriers ready
    wait_prior_grid();  // the scan kernel's prefixes and the status words
    if (status[7] == kNoSegment) return;  // the one-pass kernel decoded everything
    const bool aligned = (reinterpret_cast<uintptr_t>(src) & 15u) == 0;
    unsigned long long* timeout = status + 4;
    const LineLayout ly{uint32_t(status[6])};
    const uint64_t GW = uint64_t(gridDim.x) * kWarps;

    // Starts the bulk copy of a whole, aligned segment into buffer k; false if
    // the segment is staged with plain loads instead.
    auto issue = [&](uint64_t seg, int k) -> bool {
        const uint64_t base = seg * kSeg;
        if (!aligned || m - base < kSeg) return false;
        if (lane == 0) {
            mbar_arrive_expect_tx(&bars[warp][k], kSeg);
            bulk_load(bufs[warp][k] + kLead, src + base, kSeg, &bars[warp][k]);
        }
        return true;
    };

    uint32_t phases = 0;
    uint64_t seg = uint64_t(blockIdx.x) * kWarps + warp;
    int k = 0;
    bool by_copy = seg < nseg ? issue(seg, 0) : false;
    // the segment's raw start as lk ly.Q + lr, stepped by dk ly.Q + dr
    uint64_t lk = 0, dk = 0;
    uint32_t lr = 0, dr = 0;
    if (ly.L) {
        lk = seg * kSeg / ly.Q;
        lr = uint32_t(seg * kSeg - lk * ly.Q);
        dk = GW * kSeg / ly.Q;
        dr = uint32_t(GW * kSeg - dk * ly.Q);
    }
    for (; seg < nseg; seg += GW, k ^= 1) {
        const uint64_t next = seg + GW;
        fence_proxy_async_smem();  // this lane's accesses to buffer k^1 before the copy below
        __syncwarp();
        const bool next_by_copy = next < nseg ? issue(next, k ^ 1) : false;
        uint8_t* buf = bufs[warp][k];
        const uint64_t base = seg * kSeg;
        const uint32_t len = uint32_t(m - base < kSeg ? m - base : kSeg);
        if (by_copy) {
            const bool ok =
                __all_sync(0xffffffffu, wait_copy(&bars[warp][k], (phases >> k) & 1u, wait_limit_ns));
            phases ^= 1u << k;
            if (!ok) {
                if (next_by_copy)  // let the copy in flight land before the block can exit
                    wait_copy(&bars[warp][k ^ 1], (phases >> (k ^ 1)) & 1u, wait_limit_ns);
                if (lane == 0) {
                    atomicExch(timeout, 1ull);
                    atomicOr(&g_fault, 1u);
                }
                return;
            }
        } else {
            uint4 v[kRows];
            load_rows(src + base, len, aligned, lane, v);
#pragma unroll
            for (int r = 0; r < kRows; ++r)
                *reinterpret_cast<uint4*>(buf + kLead + kRow * r + 16 * lane) = v[r];
            __syncwarp();
        }
        const uint64_t pre = states[seg], blk = totals[seg / kSegsPerBlock];
        const uint64_t P = st_count(blk) + st_count(pre);
        const uint32_t prev_last = st_flag(pre) ? st_last(pre) : st_flag(blk) ? st_last(blk) : 0u;

        const LinesResult fast =
            ly.L && len == kSeg
                ? decode_segment_lines(buf, lut, lane, ly, lk, lr, P, prev_last, dst)
                : kLinesNo;
        lk += dk;
        lr += dr;
        if (lr >= ly.Q) {
            lr -= ly.Q;
            ++lk;
        }
        if (fast != kLinesDone) {
            if (fast == kLinesSpoilt || fast == kLinesIrregular) {  // stage the segment again
                uint4 v[kRows];
                load_rows(src + base, len, aligned, lane, v);
#pragma unroll
                for (int r = 0; r < kRows; ++r)
                    *reinterpret_cast<uint4*>(buf + kLead + kRow * r + 16 * lane) = v[r];
                __syncwarp();
            }
            decode_segment(buf, lut, flags, lane, P, prev_last, base, dst, status);
        }
        by_copy = next_by_copy;
    }
}

// ---------------------------------------------------------------- 0. one pass
// Inputs laid out as lines of L data characters and a fixed break (the layout
// of the first line, as the scan kernel detects it): the data characters
// before a segment that starts at raw position k Q + r are then P = k L +
// min(r, L), with no count, so every segment is decoded from one read of the
// input. Each whole segment takes the line-layout fast path with that P;
// the path also tells a segment whose whitespace sits elsewhere than the
// layout's breaks (kLinesIrregular) from one that only holds bad bytes or '='
// (kLinesSpoilt, decoded by the general path with the same P). The last,
// shorter segment is checked byte by byte against the layout and decoded by
// the general path. The first irregular segment is recorded in status[7]:
// its own P is right, but those of later segments may not be, so the count,
// scan and decode kernels then decode the whole input again. Without a
// layout status[7] = 0 at once. The one-pass kernel writes output only at
// the positions its P gives, inside b64_decoded_max_length(m).
__device__ __forceinline__ uint32_t block_line_layout(const uint8_t* __restrict__ src, uint64_t m,
                                                      uint32_t* s_first, uint32_t* s_word) {
    const int tid = threadIdx.x;
    if (tid == 0) *s_first = kScanThreads;
    __syncthreads();
    for (int i = tid; i < kScanThreads; i += blockDim.x) {
        if (uint64_t(i) < m) {
            const uint32_t c = src[i];
            if (c == '\r' || c == '\n' || c == ' ') atomicMin(s_first, uint32_t(i));
        }
    }
    __syncthreads();
    if (tid == 0) *s_word = line_layout_word(src, m, *s_first);
    __syncthreads();
    return *s_word;
}

// Whether the whitespace of a segment's first len bytes (staged at raw,
// starting at layout column r of its line) is exactly at the layout's
// break positions. Warp-collective.
__device__ __forceinline__ bool segment_fits_layout(const uint8_t* raw, uint32_t len,
                                                    const LineLayout& ly, uint32_t r, int lane) {
    bool ok = true;
    for (uint32_t i = lane; i < len; i += 32) {
        const uint32_t col = (r + i) % ly.Q;
        const uint32_t c = raw[i];
        const bool space = c == '\r' || c == '\n' || c == ' ';
        if (space != (col >= ly.L)) ok = false;
    }
    return __all_sync(0xffffffffu, ok);
}

__global__ void __launch_bounds__(kThreads, 6)
    mime_onepass_kernel(const uint8_t* __restrict__ src, uint64_t m, uint8_t* __restrict__ dst,
                        const __grid_constant__ DecodeTable tab, int flags,
                        unsigned long long* __restrict__ status, uint64_t nseg,
                        uint64_t wait_limit_ns) {
    __shared__ __align__(256) uint8_t lut[256];  // 0..63, 0x80 (bad or '='), kSpace
    __shared__ __align__(16) uint8_t bufs[kWarps][2][kBuf];
    __shared__ uint64_t bars[kWarps][2];
    __shared__ uint32_t s_first, s_word;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < 64; i += kThreads) reinterpret_cast<uint32_t*>(lut)[i] = tab.w[i];
    if (lane == 0) {
        mbar_init(&bars[warp][0], 1);
        mbar_init(&bars[warp][1], 1);
        fence_mbar_init();
    }
    const uint32_t word = block_line_layout(src, m, &s_first, &s_word);  // synchronises
    if (tid == 0) lut['\r'] = lut['\n'] = lut[' '] = uint8_t(kSpace);
    wait_prior_grid();  // the status words are initialised
    if (blockIdx.x == 0 && tid == 0) status[6] = word;
    if (!word) {  // no layout: the counting path decodes everything
        if (blockIdx.x == 0 && tid == 0) atomicMin(status + 7, 0ull);
        return;
    }
    __syncthreads();  // the table's whitespace entries
    const LineLayout ly{word};
    const bool aligned = (reinterpret_cast<uintptr_t>(src) & 15u) == 0;
    const uint64_t GW = uint64_t(gridDim.x) * kWarps;

    // Whole aligned segments come by one bulk copy, with the 16 bytes before
    // the segment (they hold the data byte before it) in the buffer's lead.
    auto issue = [&](uint64_t seg, int k) -> bool {
        const uint64_t base = seg * kSeg;
        if (!aligned || m - base < kSeg) return false;
        if (lane == 0) {
            const uint32_t lead = seg ? kLead : 0u;
            mbar_arrive_expect_tx(&bars[warp][k], kSeg + lead);
            bulk_load(bufs[warp][k] + kLead - lead, src + base - lead, kSeg + lead,
                      &bars[warp][k]);
        }
        return true;
    };
    auto stage_plain = [&](uint8_t* buf, uint64_t base, uint32_t len, bool lead) {
        uint4 v[kRows];
        load_rows(src + base, len, aligned, lane, v);
#pragma unroll
        for (int r = 0; r < kRows; ++r)
            *reinterpret_cast<uint4*>(buf + kLead + kRow * r + 16 * lane) = v[r];
        if (lead && lane < int(kLead)) buf[lane] = src[base - kLead + lane];
        __syncwarp();
    };

    uint32_t phases = 0;
    uint64_t seg = uint64_t(blockIdx.x) * kWarps + warp;
    int k = 0;
    bool by_copy = seg < nseg ? issue(seg, 0) : false;
    // the segment's raw start as lk ly.Q + lr, stepped by dk ly.Q + dr
    uint64_t lk = seg * kSeg / ly.Q;
    uint32_t lr = uint32_t(seg * kSeg - lk * ly.Q);
    const uint64_t dk = GW * kSeg / ly.Q;
    const uint32_t dr = uint32_t(GW * kSeg - dk * ly.Q);
    for (; seg < nseg; seg += GW, k ^= 1) {
        const uint64_t next = seg + GW;
        fence_proxy_async_smem();  // this lane's accesses to buffer k^1 before the copy below
        __syncwarp();
        const bool next_by_copy = next < nseg ? issue(next, k ^ 1) : false;
        uint8_t* buf = bufs[warp][k];
        const uint64_t base = seg * kSeg;
        const uint32_t len = uint32_t(m - base < kSeg ? m - base : kSeg);
        if (by_copy) {
            const bool ok = __all_sync(0xffffffffu,
                                       wait_copy(&bars[warp][k], (phases >> k) & 1u, wait_limit_ns));
            phases ^= 1u << k;
            if (!ok) {
                if (next_by_copy)  // let the copy in flight land before the block can exit
                    wait_copy(&bars[warp][k ^ 1], (phases >> (k ^ 1)) & 1u, wait_limit_ns);
                if (lane == 0) {
                    atomicExch(status + 4, 1ull);
                    atomicOr(&g_fault, 1u);
                }
                return;
            }
        } else {
            stage_plain(buf, base, len, seg > 0);
        }
        // the layout's count before the segment, and its last data byte
        const uint64_t P = lk * ly.L + (lr < ly.L ? lr : ly.L);
        const uint32_t back = lr == 0 ? 1 + ly.eol : lr > ly.L ? lr - ly.L + 1 : 1u;
        const uint32_t prev_last = P ? buf[kLead - back] : 0u;
        bool irregular = false, general = false;
        if (len == kSeg) {
            const LinesResult r =
                decode_segment_lines(buf, lut, lane, ly, lk, lr, P, prev_last, dst);
            irregular = r == kLinesIrregular || r == kLinesNo;
            if (r == kLinesSpoilt) {  // bad bytes or '=': the general path, same P
                stage_plain(buf, base, len, false);
                general = true;
            }
        } else {
            irregular = !segment_fits_layout(buf + kLead, len, ly, lr, lane);
            general = !irregular;
        }
        // one call site, so the kernel holds one copy of the general path
        if (general) decode_segment(buf, lut, flags, lane, P, prev_last, base, dst, status);
        if (irregular && lane == 0) atomicMin(status + 7, (unsigned long long)seg);
        lk += dk;
        lr += dr;
        if (lr >= ly.Q) {
            lr -= ly.Q;
            ++lk;
        }
        by_copy = next_by_copy;
    }
}

// ---------------------------------------------------------------- 4. finalize
// The padding and length rules on a document's compacted stream (and, in
// canonical mode, the unused bits of a partial final group's last data
// character, found by walking back over the trailing whitespace and padding).
// whole: the document's state (data characters, last data byte); st3: its
// status words (first bad byte, first '=' raw and compacted).
__device__ int64_t mime_result(const uint8_t* __restrict__ src, uint64_t m, int flags,
                               const DecodeTable& tab, uint64_t whole,
                               const unsigned long long* __restrict__ st3) {
    const bool padded = flags & 1, canonical = flags & 2;
    const uint64_t mc = st_count(whole);  // data characters
    const uint32_t last = st_last(whole);
    uint64_t err = st3[0];
    uint64_t pads = 0;
    if (padded && st3[2] != kNoError) {
        const uint64_t qe = st3[2];
        const bool ok = qe + 1 == mc || (qe + 2 == mc && last == '=');
        if (ok) pads = mc - qe;
        else err = st3[1] < err ? st3[1] : err;
    }
    if (padded ? (mc % 4 != 0) : (mc % 4 == 1)) err = m < err ? m : err;
    const uint64_t d = mc - pads;
    if (canonical && (d % 4 == 2 || d % 4 == 3)) {
        // raw position of data character d - 1: the (pads + 1)-th data
        // character from the end
        uint64_t p = m, seen = 0;
        while (p > 0) {
            const uint32_t ch = src[--p];
            if (ch == '\r' || ch == '\n' || ch == ' ') continue;
            if (++seen == pads + 1) break;
        }
        const uint32_t v = (tab.w[src[p] >> 2] >> (8 * (src[p] & 3))) & 0xFFu;
        const uint32_t low = d % 4 == 2 ? 15u : 3u;
        if (!(v & kBad) && (v & low)) err = p < err ? p : err;
    }
    return err != kNoError ? -int64_t(err) - 1 : int64_t(bytes_for(mc - pads));
}

// One thread: the result of the single-document decode.
__global__ void mime_finalize_kernel(const uint8_t* __restrict__ src, uint64_t m, int flags,
                                     const __grid_constant__ DecodeTable tab,
                                     const unsigned long long* __restrict__ status,
                                     int64_t* __restrict__ d_result) {
    wait_prior_grid();  // every kernel before it has completed
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (status[4]) {
        *d_result = B64_E_TIMEOUT;
        return;
    }
    uint64_t whole = status[5];
    if (status[7] == kNoSegment && status[6]) {
        // one pass, every segment in the layout: the data characters and the
        // last one follow from it
        const LineLayout ly{uint32_t(status[6])};
        const uint64_t k = m / ly.Q, r = m - k * ly.Q;
        const uint64_t mc = k * ly.L + (r < ly.L ? r : ly.L);
        const uint64_t j = mc - 1;
        const uint32_t last = mc ? src[j / ly.L * ly.Q + j % ly.L] : 0u;
        whole = make_state(mc != 0, last, mc);
    }
    *d_result = mime_result(src, m, flags, tab, whole, status);
}

// ---------------------------------------------------------------- batched documents
// Document d is bytes [src_off[d], src_off[d+1]) of src, decoded to
// dst + dst_off[d] with its own alphabet, exactly as the single-document call
// decodes it. Its ceil(len / kSeg) segments keep their state words at slots
// doc_slot(d) + k, doc_slot(d) = (src_off[d] - src_off[0]) / kSeg + d: the
// slot ranges of consecutive documents never overlap (the next document's
// first slot lies at least ceil(len / kSeg) further on), so no scan over the
// documents is needed and a slot's document is found by a search. Launch
// sequence: memset of the documents' status words; one warp per document
// detecting its line layout; the one-pass decode of the documents with one
// (each segment with the count the layout gives it, a segment off the layout
// marking its document); then, for the documents without a layout or marked,
// count, one warp per document scanning its segments (and clearing its
// status words), decode; one thread per document for the result. Documents start anywhere, so a segment is
// staged by one bulk copy of the 16-byte aligned span around it (plain
// aligned loads where that span would leave the batch's input) and read
// through a funnel shift; the wait on each copy is bounded in time, and a
// document one of whose copies timed out gets B64_E_TIMEOUT.
__device__ __forceinline__ uint64_t doc_slot(const int64_t* __restrict__ src_off, int64_t d) {
    return uint64_t(src_off[d] - src_off[0]) / kSeg + uint64_t(d);
}

// Warp-cooperative: the largest d in [0, n) with doc_slot(d) <= g (n >= 1).
__device__ int64_t warp_find_doc(const int64_t* __restrict__ src_off, int64_t n, uint64_t g,
                                 int lane) {
    int64_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const int64_t step = (hi - lo + 31) / 32;
        const int64_t probe = lo + int64_t(lane) * step;
        const bool le = probe < hi && doc_slot(src_off, probe) <= g;
        const uint32_t mask = __ballot_sync(0xffffffffu, le);
        const int k = 31 - __clz(mask);  // lane 0 always holds (probe = lo)
        const int64_t nlo = lo + int64_t(k) * step;
        hi = nlo + step < hi ? nlo + step : hi;
        lo = nlo;
    }
    return lo;
}

// 16 bytes at p + off (bytes at or past len read as spaces). Aligned 16-byte
// loads and a funnel shift when both aligned blocks lie inside [lo, hi) (the
// batch's input); byte loads otherwise.
__device__ __forceinline__ uint4 load_chunk_any(const uint8_t* p, uint32_t off, uint32_t len,
                                                const uint8_t* lo, const uint8_t* hi) {
    const uint8_t* q = p + off;
    if (off + 16 <= len) {
        const uintptr_t a = reinterpret_cast<uintptr_t>(q);
        const uint32_t sh = uint32_t(a & 15);
        if (sh == 0) return *reinterpret_cast<const uint4*>(q);
        const uint8_t* a0 = reinterpret_cast<const uint8_t*>(a & ~uintptr_t(15));
        if (a0 >= lo && a0 + 32 <= hi) {
            const uint4 x = *reinterpret_cast<const uint4*>(a0);
            const uint4 y = *reinterpret_cast<const uint4*>(a0 + 16);
            const uint32_t sb = 8 * (sh & 3);
            auto f = [sb](uint32_t a, uint32_t b, uint32_t c, uint32_t d, uint32_t e) {
                return make_uint4(__funnelshift_r(a, b, sb), __funnelshift_r(b, c, sb),
                                  __funnelshift_r(c, d, sb), __funnelshift_r(d, e, sb));
            };
            switch (sh >> 2) {  // the same in every lane of the segment
                case 0: return f(x.x, x.y, x.z, x.w, y.x);
                case 1: return f(x.y, x.z, x.w, y.x, y.y);
                case 2: return f(x.z, x.w, y.x, y.y, y.z);
                default: return f(x.w, y.x, y.y, y.z, y.w);
            }
        }
    }
    uint4 v;
    uint8_t* b = reinterpret_cast<uint8_t*>(&v);
    for (int k = 0; k < 16; ++k) b[k] = off + k < len ? q[k] : uint8_t(' ');
    return v;
}

struct DocSeg {
    int64_t d;         // document
    uint64_t k;        // segment within it
    uint32_t len;      // bytes of the segment
    const uint8_t* p;  // its first byte
};

__device__ __forceinline__ uint64_t doc_slots(const int64_t* __restrict__ src_off, int64_t n) {
    return uint64_t(src_off[n] - src_off[0]) / kSeg + uint64_t(n) + 1;
}

// A warp's walk over its own contiguous range of slots [g0, g1): the
// document of the last slot found is remembered, so the 32-way document
// search runs once per document the range touches instead of once per slot.
// status word 0 of a document whose bulk copy did not arrive (offsets are
// below 2^62): its result becomes B64_E_TIMEOUT
constexpr uint64_t kDocTimedOut = uint64_t(1) << 62;

// Bit 32 of a document's line word (line_docs): its segments need the
// counting passes (it has no line layout, or a segment broke it); bits 0..31:
// the layout word.
constexpr uint64_t kDocCounted = uint64_t(1) << 32;

struct SlotWalk {
    uint64_t g, g1;
    int64_t d = -1;                  // the remembered document
    uint64_t first = 0, nseg = 0;    // its first slot and its segments
    // with line_docs: only the documents whose kDocCounted bit equals counted
    const unsigned long long* line_docs = nullptr;
    bool counted = false;
    __device__ SlotWalk(uint64_t nslots, uint64_t warp, uint64_t warps) {
        const uint64_t per = (nslots + warps - 1) / warps;
        g = warp * per < nslots ? warp * per : nslots;
        g1 = g + per < nslots ? g + per : nslots;
    }
    // The next used slot of the range (its segment in *ds, its slot in *slot);
    // false when the range is done. Warp-collective.
    __device__ bool next(const uint8_t* src, const int64_t* __restrict__ src_off, int64_t n,
                         int lane, DocSeg* ds, uint64_t* slot) {
        for (; g < g1; ++g) {
            if (d < 0 || g < first || g >= first + nseg) {
                if (d >= 0 && g >= first + nseg && d + 1 < n && g < doc_slot(src_off, d + 1))
                    continue;  // a slot between the remembered document and the next
                d = warp_find_doc(src_off, n, g, lane);
                first = doc_slot(src_off, d);
                nseg = (uint64_t(src_off[d + 1] - src_off[d]) + kSeg - 1) / kSeg;
                if (line_docs && ((line_docs[d] & kDocCounted) != 0) != counted)
                    nseg = 0;                     // not this pass's document: skip its slots
                if (g >= first + nseg) continue;  // an unused slot
            }
            const uint64_t k = g - first;
            const uint64_t len = uint64_t(src_off[d + 1] - src_off[d]);
            ds->d = d;
            ds->k = k;
            ds->len = uint32_t(len - k * kSeg < kSeg ? len - k * kSeg : kSeg);
            ds->p = src + src_off[d] + k * kSeg;
            *slot = g++;
            return true;
        }
        return false;
    }
};

__global__ void __launch_bounds__(kCountThreads, 4)
    mime_count_docs_kernel(const uint8_t* __restrict__ src, const int64_t* __restrict__ src_off,
                           int64_t n, unsigned long long* __restrict__ states,
                           const unsigned long long* __restrict__ line_docs,
                           const unsigned long long* __restrict__ none_counted,
                           uint64_t slot_cap) {
    const int lane = threadIdx.x & 31;
    wait_prior_grid();  // line_docs and none_counted are written by the kernels before
    if (*none_counted) return;  // every document kept its line layout
    const uint64_t nslots = doc_slots(src_off, n);
    if (nslots > slot_cap) return;  // workspace too small: the results say so
    const uint64_t gw = (uint64_t(blockIdx.x) * kCountThreads + threadIdx.x) >> 5;
    const uint64_t GW = (uint64_t(gridDim.x) * kCountThreads) >> 5;
    const uint8_t* lo = src + src_off[0];
    const uint8_t* hi = src + src_off[n];
    SlotWalk walk(nslots, gw, GW);
    walk.line_docs = line_docs;  // the documents the one-pass kernel left to this path
    walk.counted = true;
    DocSeg ds;
    uint64_t g;
    while (walk.next(src, src_off, n, lane, &ds, &g)) {
        uint32_t key = 0;
        uint4 v[kRows];
#pragma unroll
        for (int r = 0; r < kRows; ++r) v[r] = load_chunk_any(ds.p, kRow * r + 16 * lane, ds.len, lo, hi);
        const uint32_t count = __reduce_add_sync(0xffffffffu, rows_count(v, lane, &key));
        key = __reduce_max_sync(0xffffffffu, key);
        if (lane == 0) states[g] = make_state(key != 0, key & 0xFFu, count);
    }
}

// One warp per document the counting passes decode (kDocCounted): its
// segments' states become prefixes (data characters and last data byte before
// the segment, within the document); doc_state[d] = the whole document's; its
// status words, which the one-pass kernel may have set from layout counts,
// return to "none" for the decode that follows.
__global__ void __launch_bounds__(256)
    mime_scan_docs_kernel(const uint8_t* __restrict__ src, const int64_t* __restrict__ src_off,
                          int64_t n, unsigned long long* __restrict__ states,
                          unsigned long long* __restrict__ doc_state,
                          const unsigned long long* __restrict__ line_docs,
                          unsigned long long* __restrict__ status_docs,
                          const unsigned long long* __restrict__ none_counted,
                          uint64_t slot_cap) {
    const int lane = threadIdx.x & 31;
    wait_prior_grid();
    if (*none_counted) return;
    if (doc_slots(src_off, n) > slot_cap) return;
    const int64_t gw = (int64_t(blockIdx.x) * 256 + threadIdx.x) >> 5;
    const int64_t GW = (int64_t(gridDim.x) * 256) >> 5;
    for (int64_t d = gw; d < n; d += GW) {
        if (!(line_docs[d] & kDocCounted)) continue;
        if (lane < 3 && status_docs[3 * d + lane] != kDocTimedOut)
            status_docs[3 * d + lane] = ~0ull;
        const uint64_t first = doc_slot(src_off, d);
        const uint64_t segs = (uint64_t(src_off[d + 1] - src_off[d]) + kSeg - 1) / kSeg;
        uint64_t carry = 0, carry_key = 0;  // key: (segment + 1) << 8 | last byte
        for (uint64_t c = 0; c < segs; c += 32) {
            const uint64_t k = c + lane;
            const uint64_t st = k < segs ? states[first + k] : 0;
            const uint64_t cnt = st_count(st);
            const uint64_t key = st_flag(st) ? ((k + 1) << 8) | st_last(st) : 0;
            uint64_t incl = cnt, kincl = key;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t u = __shfl_up_sync(0xffffffffu, incl, o);
                const uint64_t uk = __shfl_up_sync(0xffffffffu, kincl, o);
                if (lane >= o) {
                    incl += u;
                    kincl = uk > kincl ? uk : kincl;
                }
            }
            uint64_t kex = __shfl_up_sync(0xffffffffu, kincl, 1);
            if (lane == 0) kex = 0;
            kex = kex > carry_key ? kex : carry_key;
            if (k < segs) states[first + k] = make_state(kex != 0, uint32_t(kex & 0xFFu), carry + incl - cnt);
            carry += __shfl_sync(0xffffffffu, incl, 31);
            const uint64_t top = __shfl_sync(0xffffffffu, kincl, 31);
            carry_key = top > carry_key ? top : carry_key;
        }
        if (lane == 0) doc_state[d] = make_state(carry_key != 0, uint32_t(carry_key & 0xFFu), carry);
    }
}

// One warp per document: its line layout (as the single-document call
// detects it, from the first 1024 bytes) into line_docs[d], with kDocCounted
// set when there is none; for a document with a layout, doc_state[d] = the
// data characters and last data byte the layout gives (the finalize kernel's
// figures if every segment keeps to it; the scan kernel replaces them
// otherwise).
__global__ void __launch_bounds__(256)
    mime_layout_docs_kernel(const uint8_t* __restrict__ src, const int64_t* __restrict__ src_off,
                            int64_t n, unsigned long long* __restrict__ line_docs,
                            unsigned long long* __restrict__ doc_state,
                            unsigned long long* __restrict__ none_counted, uint64_t slot_cap) {
    const int lane = threadIdx.x & 31;
    if (doc_slots(src_off, n) > slot_cap) return;
    const int64_t gw = (int64_t(blockIdx.x) * 256 + threadIdx.x) >> 5;
    const int64_t GW = (int64_t(gridDim.x) * 256) >> 5;
    for (int64_t d = gw; d < n; d += GW) {
        const uint8_t* p = src + src_off[d];
        const uint64_t len = uint64_t(src_off[d + 1] - src_off[d]);
        uint32_t c[kScanThreads / 32];  // all loads issued before any is used
#pragma unroll
        for (int j = 0; j < kScanThreads / 32; ++j) {
            const uint32_t i = uint32_t(lane) + 32 * j;
            c[j] = i < len ? p[i] : 0u;
        }
        uint32_t f = kScanThreads;
#pragma unroll
        for (int j = kScanThreads / 32 - 1; j >= 0; --j)
            if (c[j] == '\r' || c[j] == '\n' || c[j] == ' ') f = uint32_t(lane) + 32 * j;
        f = __reduce_min_sync(0xffffffffu, f);
        if (lane == 0) {
            const uint32_t word = line_layout_word(p, len, f);
            line_docs[d] = word ? uint64_t(word) : kDocCounted;
            if (!word) *none_counted = 0;
            if (word) {
                const LineLayout ly{word};
                const uint64_t k = len / ly.Q, r = len - k * ly.Q;
                const uint64_t mc = k * ly.L + (r < ly.L ? r : ly.L);
                const uint64_t j = mc - 1;
                const uint32_t last = mc ? p[j / ly.L * ly.Q + j % ly.L] : 0u;
                doc_state[d] = make_state(mc != 0, last, mc);
            }
        }
    }
}

constexpr int kDocWarps = 4;
// Blocks an SM the register bound of the one-pass documents kernel aims at
#ifndef B64_MIME_DOCS_ONEPASS_BLOCKS
#define B64_MIME_DOCS_ONEPASS_BLOCKS 5
#endif
// a segment's 16-byte aligned span (at most kSeg + 32 bytes) fits a buffer after its lead
static_assert(kLead + kSeg + 32 <= kBuf, "document staging");

// A segment's raw start S in its document's line layout as line * Q +
// column: the line, by a 32-bit division where S < 2^32.
__device__ __forceinline__ uint64_t line_of(uint64_t S, uint32_t Q) {
    return (S >> 32) ? S / Q : uint64_t(uint32_t(S) / Q);
}

// Starts the bulk copy of the 16-byte aligned span around a document
// segment's bytes into stage (byte 0 of the segment lands at
// stage[p & 15]); false (nothing started) when the span would leave the
// batch's input [lo, hi). Lane 0 only.
__device__ __forceinline__ bool issue_doc_segment(uint8_t* stage, const DocSeg& ds,
                                                  const uint8_t* lo, const uint8_t* hi,
                                                  uint64_t* bar) {
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(ds.p) & ~uintptr_t(15);
    const uintptr_t a1 = (reinterpret_cast<uintptr_t>(ds.p) + ds.len + 15) & ~uintptr_t(15);
    if (a0 < reinterpret_cast<uintptr_t>(lo) || a1 > reinterpret_cast<uintptr_t>(hi)) return false;
    mbar_arrive_expect_tx(bar, uint32_t(a1 - a0));
    bulk_load(stage, reinterpret_cast<const void*>(a0), uint32_t(a1 - a0), bar);
    return true;
}

// kOnePass: the documents with a line layout (kDocCounted clear), every
// segment decoded with the data count the layout gives it (as the
// single-document one-pass kernel does); a segment off the layout sets its
// document's kDocCounted. Otherwise: the kDocCounted documents, with the
// counts of the count and scan kernels.
template <bool kOnePass>
__global__ void __launch_bounds__(32 * kDocWarps, kOnePass ? B64_MIME_DOCS_ONEPASS_BLOCKS : 5)
    mime_decode_docs_kernel(const uint8_t* __restrict__ src, const int64_t* __restrict__ src_off,
                            int64_t n, uint8_t* __restrict__ dst,
                            const int64_t* __restrict__ dst_off,
                            const __grid_constant__ BatchTables tabs,
                            const uint8_t* __restrict__ alph_id,
                            unsigned long long* __restrict__ status_docs,
                            unsigned long long* __restrict__ line_docs,
                            const unsigned long long* __restrict__ states,
                            unsigned long long* __restrict__ none_counted, uint64_t slot_cap) {
    __shared__ __align__(256) uint8_t luts[kMaxAlphabets][256];  // 0..63, 0x80, kSpace
    __shared__ __align__(16) uint8_t bufs[kDocWarps][2][kBuf];
    __shared__ uint64_t bars[kDocWarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < kMaxAlphabets * 64; i += 32 * kDocWarps)
        reinterpret_cast<uint32_t*>(luts)[i] = tabs.dec[i / 64].w[i % 64];
    __syncthreads();
    if (tid < kMaxAlphabets) luts[tid]['\r'] = luts[tid]['\n'] = luts[tid][' '] = uint8_t(kSpace);
    if (lane == 0) {
        mbar_init(&bars[warp], 1);
        fence_mbar_init();
    }
    __syncthreads();
    wait_prior_grid();  // the layout words, states and status words of the kernels before
    if constexpr (!kOnePass) {
        if (*none_counted) return;  // every document kept its line layout
    }
    const uint64_t nslots = doc_slots(src_off, n);
    if (nslots > slot_cap) return;
    const uint8_t* lo = src + src_off[0];
    const uint8_t* hi = src + src_off[n];
    const uint64_t GW = uint64_t(gridDim.x) * kDocWarps;

    SlotWalk walk(nslots, uint64_t(blockIdx.x) * kDocWarps + warp, GW);
    walk.line_docs = line_docs;
    walk.counted = !kOnePass;
    // Slot g's segment arrives in one of the warp's two buffers by a bulk copy
    // of its aligned span (segment byte i at buf[kLead + (p & 15) + i]),
    // started while the slot before it is decoded in the other buffer. The
    // line path decodes it there; otherwise it is first moved down to
    // buf + kLead.
    uint64_t g = 0;
    DocSeg ds;
    bool have = walk.next(src, src_off, n, lane, &ds, &g), by_copy = false;
    int kb = 0;  // the buffer of slot g
    if (have && lane == 0) by_copy = issue_doc_segment(bufs[warp][0] + kLead, ds, lo, hi, &bars[warp]);
    by_copy = __shfl_sync(0xffffffffu, by_copy, 0);
    // A slot's document metadata (alphabet, layout word, output offset; the
    // one-pass kernel's data byte before the segment, the other's segment
    // state), loaded with the slot's copy so the loads overlap the slot
    // before it.
    struct SegMeta {
        uint64_t pre;
        int64_t out;
        uint32_t word, prev;
        int a;
    };
    auto fetch = [&](const DocSeg& d, uint64_t slot) {
        SegMeta m;
        m.a = alph_id ? (alph_id[d.d] & (kMaxAlphabets - 1)) : 0;
        m.word = uint32_t(line_docs[d.d]);
        m.out = dst_off[d.d];
        m.pre = 0;
        m.prev = 0;
        if constexpr (kOnePass) {
            // the data byte before the segment (every segment but a
            // document's first has one): the byte before it, or the last
            // before the break where the segment starts a line or inside
            // the break
            const uint32_t L = m.word & 0xFFFFu, eol = m.word >> 16, Q = L + eol;
            if (d.k && L) {
                const uint64_t S = d.k * kSeg;
                const uint32_t lr = uint32_t(S - line_of(S, Q) * Q);
                const uint32_t back = lr == 0 ? 1 + eol : lr > L ? lr - L + 1 : 1u;
                m.prev = d.p[-int64_t(back)];
            }
        } else {
            m.pre = states[slot];
        }
        return m;
    };
    SegMeta meta{};
    if (have) meta = fetch(ds, g);
    uint32_t phase = 0;
    while (have) {
        unsigned long long* st3 = status_docs + 3 * ds.d;
        uint8_t* const buf = bufs[warp][kb];
        const LineLayout ly{meta.word};
        auto stage_plain = [&] {
#pragma unroll
            for (int r = 0; r < kRows; ++r) {
                const uint32_t off = kRow * r + 16 * lane;
                *reinterpret_cast<uint4*>(buf + kLead + off) =
                    load_chunk_any(ds.p, off, ds.len, lo, hi);
            }
            __syncwarp();
        };
        uint32_t delta = 0;  // the segment's first byte is at buf[kLead + delta]
        if (by_copy) {
            const bool ok = __all_sync(0xffffffffu, wait_copy(&bars[warp], phase, kWaitLimitNs));
            phase ^= 1u;
            if (!ok) {
                if (lane == 0) {
                    atomicMin(st3, (unsigned long long)kDocTimedOut);
                    atomicOr(&g_fault, 1u);
                    // give the copy one more bounded wait to land before the
                    // block can exit (its stage buffer belongs to the block)
                    wait_copy(&bars[warp], phase ^ 1u, kWaitLimitNs);
                }
                return;
            }
            const uint32_t pd = uint32_t(reinterpret_cast<uintptr_t>(ds.p) & 15);
            if (ds.len == kSeg && ly.L >= 16 && (ly.eol == 1 || (pd & 1u) == 0)) {
                delta = pd;  // the line path reads the segment where it landed
            } else if (pd || ds.len < kSeg) {
                // moved down by pd, a row at a time (a row's reads reach 16
                // bytes into the next lane's row part, so all come before its
                // writes; the next row's reads start past them); bytes at or
                // past len read as spaces
                uint8_t* const raw = buf + kLead;
#pragma unroll
                for (int r = 0; r < kRows; ++r) {
                    const uint32_t off = kRow * r + 16 * lane;
                    uint4 v;
                    if (off + 16 <= ds.len) {
                        v = load16_shifted_u(raw, pd + off);
                    } else {
                        uint8_t* bv = reinterpret_cast<uint8_t*>(&v);
                        for (int j = 0; j < 16; ++j)
                            bv[j] = off + j < ds.len ? raw[pd + off + j] : uint8_t(' ');
                    }
                    __syncwarp();
                    *reinterpret_cast<uint4*>(raw + off) = v;
                }
            }
        } else {
            stage_plain();
        }
        // this lane's accesses to the other buffer (the slot before) come
        // before the next slot's copy into it
        fence_proxy_async_smem();
        __syncwarp();
        uint64_t g2 = 0;
        DocSeg ds2;
        const bool have2 = walk.next(src, src_off, n, lane, &ds2, &g2);
        bool by_copy2 = false;
        if (have2 && lane == 0)
            by_copy2 = issue_doc_segment(bufs[warp][kb ^ 1] + kLead, ds2, lo, hi, &bars[warp]);
        by_copy2 = __shfl_sync(0xffffffffu, by_copy2, 0);
        SegMeta meta2{};
        if (have2) meta2 = fetch(ds2, g2);
        const int a = meta.a;
        const int flags = (tabs.padded[a] ? 1 : 0) | (tabs.canonical[a] ? 2 : 0);
        const uint64_t S = ds.k * kSeg, lk = ly.L ? line_of(S, ly.Q) : 0;
        const uint32_t lr = uint32_t(S - lk * ly.Q);
        uint8_t* const out_doc = dst + meta.out;
        if constexpr (kOnePass) {
            // the layout's count before the segment, and its last data byte
            const uint64_t P = lk * ly.L + (lr < ly.L ? lr : ly.L);
            const uint32_t prev_last = meta.prev;
            bool irregular = false, general = false;
            if (ds.len == kSeg) {
                const LinesResult r = decode_segment_lines(buf, luts[a], lane, ly, lk, lr, P,
                                                           prev_last, out_doc, delta);
                irregular = r == kLinesIrregular || r == kLinesNo;
                if (r == kLinesSpoilt) {  // bad bytes or '=': the general path, same P
                    stage_plain();
                    general = true;
                }
            } else {
                irregular = !segment_fits_layout(buf + kLead, ds.len, ly, lr, lane);
                general = !irregular;
            }
            // one call site, so the kernel holds one copy of the general path
            if (general) decode_segment(buf, luts[a], flags, lane, P, prev_last, S, out_doc, st3);
            if (irregular && lane == 0) {
                atomicOr(&line_docs[ds.d], (unsigned long long)kDocCounted);
                *none_counted = 0;
            }
        } else {
            const uint64_t pre = meta.pre;
            const uint64_t P = st_count(pre);
            const uint32_t prev_last = st_flag(pre) ? st_last(pre) : 0u;
            LinesResult fast = kLinesNo;
            if (ly.L && ds.len == kSeg)
                fast = decode_segment_lines(buf, luts[a], lane, ly, lk, lr, P, prev_last, out_doc,
                                            delta);
            // the general path reads the segment at buf + kLead
            if (fast == kLinesSpoilt || fast == kLinesIrregular || (fast == kLinesNo && delta))
                stage_plain();
            if (fast != kLinesDone)
                decode_segment(buf, luts[a], flags, lane, P, prev_last, S, out_doc, st3);
        }
        __syncwarp();
        kb ^= 1;
        g = g2;
        ds = ds2;
        have = have2;
        by_copy = by_copy2;
        meta = meta2;
    }
}

__global__ void mime_finalize_docs_kernel(const uint8_t* __restrict__ src,
                                          const int64_t* __restrict__ src_off, int64_t n,
                                          const __grid_constant__ BatchTables tabs,
                                          const uint8_t* __restrict__ alph_id,
                                          const unsigned long long* __restrict__ status_docs,
                                          const unsigned long long* __restrict__ doc_state,
                                          uint64_t slot_cap, int64_t* __restrict__ results) {
    wait_prior_grid();
    const int64_t d = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (d >= n) return;
    if (doc_slots(src_off, n) > slot_cap) {
        results[d] = B64_E_INVAL;
        return;
    }
    if (status_docs[3 * d] == kDocTimedOut) {
        results[d] = B64_E_TIMEOUT;
        return;
    }
    const int a = alph_id ? (alph_id[d] & (kMaxAlphabets - 1)) : 0;
    const int flags = (tabs.padded[a] ? 1 : 0) | (tabs.canonical[a] ? 2 : 0);
    results[d] = mime_result(src + src_off[d], uint64_t(src_off[d + 1] - src_off[d]), flags,
                             tabs.dec[a], doc_state[d], status_docs + 3 * d);
}

// The bounded wait of the decode kernel on a bulk copy that is never issued:
// one thread arms a barrier for 16 bytes that never arrive and waits.
__global__ void selftest_wait_kernel(int64_t* __restrict__ d_result, uint64_t wait_limit_ns) {
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(&bar, 16);
    if (!wait_copy(&bar, 0, wait_limit_ns)) {
        atomicOr(&g_fault, 1u);
        *d_result = B64_E_TIMEOUT;
    } else {
        *d_result = 0;
    }
}

struct Occ {
    std::once_flag once;
    int ctas = 1;
};
Occ g_occ[64], g_op_occ[64], g_cd_occ[64], g_dd_occ[64], g_ddo_occ[64];

template <class K>
int occupancy(K kernel, int threads, Occ& occ) {
    std::call_once(occ.once, [&] {
        int c = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, kernel, threads, 0) != cudaSuccess)
            c = 1;
        occ.ctas = c > 0 ? c : 1;
    });
    return occ.ctas;
}

}  // namespace

size_t mime_workspace_bytes(uint64_t m) {
    const uint64_t nseg = (m + kSeg - 1) / kSeg;
    const uint64_t nblk = (nseg + kSegsPerBlock - 1) / kSegsPerBlock;
    return 64 + 8 * size_t(nseg + nblk);
}

// One warp: the single-document call's status words (see launch_mime_decode).
__global__ void mime_status_init_kernel(unsigned long long* __restrict__ status) {
    const int i = threadIdx.x;
    if (i < 8) status[i] = (i < 3 || i == 7) ? ~0ull : 0ull;
}

cudaError_t launch_mime_decode(const uint8_t* src, uint64_t m, uint8_t* dst,
                               const DecodeTable& tab, int flags, int64_t* d_result,
                               void* workspace, uint64_t wait_limit_ns, cudaStream_t st) {
    const uint64_t nseg = (m + kSeg - 1) / kSeg;
    const uint64_t nblk = (nseg + kSegsPerBlock - 1) / kSegsPerBlock;
    unsigned long long* status = static_cast<unsigned long long*>(workspace);
    unsigned long long* states = status + 8;
    unsigned long long* totals = states + nseg;
    // The init kernel sets status[0..2] (first bad byte, first '=' raw and
    // compacted) to "none"; status[3..6] (status[4]: the timeout word;
    // status[5]: the whole input's state; status[6]: the line layout) to zero;
    // status[7] (the first segment off the layout) to "none".
    // Every kernel after the init kernel is a programmatic dependent of the
    // one before it (it waits for that kernel before touching what it wrote),
    // so each launch overlaps the end of the kernel before; the count, scan
    // and decode kernels return at once when the one-pass kernel decoded
    // everything.
    mime_status_init_kernel<<<1, 32, 0, st>>>(status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (nseg) {
        const DeviceInfo& di = device_info();
        uint64_t grid = uint64_t(di.sm_count) *
                        occupancy(mime_onepass_kernel, kThreads, g_op_occ[di.device & 63]);
        const uint64_t need = (nseg + kWarps - 1) / kWarps;
        if (need < grid) grid = need;
        e = launch_dependent(mime_onepass_kernel, unsigned(grid), kThreads, 0, st, src, m, dst, tab,
                             flags, status, nseg, wait_limit_ns);
        if (e != cudaSuccess) return e;
        e = launch_dependent(mime_count_kernel, unsigned(nblk), kCountThreads, 0, st, src, m,
                             states, totals, nseg, status);
        if (e != cudaSuccess) return e;
        e = launch_dependent(mime_scan_kernel, 1, kScanThreads, 0, st, totals, nblk, status, src, m);
        if (e != cudaSuccess) return e;
        grid = uint64_t(di.sm_count) * occupancy(mime_decode_kernel, kThreads, g_occ[di.device & 63]);
        if (need < grid) grid = need;
        e = launch_dependent(mime_decode_kernel, unsigned(grid), kThreads, 0, st, src, m, dst, tab,
                             flags, status, states, totals, nseg, wait_limit_ns);
        if (e != cudaSuccess) return e;
    }
    return launch_dependent(mime_finalize_kernel, 1, 32, 0, st, src, m, flags, tab, status,
                            d_result);
}

cudaError_t launch_selftest_wait(int64_t* d_result, uint64_t wait_limit_ns, cudaStream_t st) {
    selftest_wait_kernel<<<1, 32, 0, st>>>(d_result, wait_limit_ns);
    return cudaGetLastError();
}

size_t mime_batch_workspace_bytes(int64_t n, uint64_t total_bytes) {
    const uint64_t slots = total_bytes / kSeg + uint64_t(n) + 1;
    return 8 * (5 * size_t(n) + 1 + size_t(slots));
}

cudaError_t launch_mime_decode_batch(const BatchArgs& a, const BatchTables& tabs, void* workspace,
                                     size_t workspace_bytes, cudaStream_t st) {
    if (a.n <= 0) return cudaSuccess;
    // [status: 3 words per document][none_counted][document states: n]
    // [line layouts: n][segment slots]; none_counted stays all ones while
    // every document keeps its line layout, and the counting passes then
    // return at once
    unsigned long long* status_docs = static_cast<unsigned long long*>(workspace);
    unsigned long long* none_counted = status_docs + 3 * a.n;
    unsigned long long* doc_state = none_counted + 1;
    unsigned long long* line_docs = doc_state + a.n;
    unsigned long long* states = line_docs + a.n;
    const uint64_t words = workspace_bytes / 8, fixed = 5 * uint64_t(a.n) + 1;
    const uint64_t slot_cap = words > fixed ? words - fixed : 0;
    cudaError_t e =
        cudaMemsetAsync(status_docs, 0xFF, (3 * size_t(a.n) + 1) * sizeof(uint64_t), st);
    if (e != cudaSuccess) return e;
    const DeviceInfo& di = device_info();
    const uint64_t scan_blocks = (uint64_t(a.n) + 7) / 8;
    const unsigned sb = unsigned(scan_blocks < uint64_t(di.sm_count) * 8 ? scan_blocks : di.sm_count * 8);
    // one pass for the documents with a line layout, then the counting passes
    // for the others (each kernel skips the documents it is not for); every
    // kernel after the layout kernel is a programmatic dependent of the one
    // before
    mime_layout_docs_kernel<<<sb, 256, 0, st>>>(a.src, a.src_off, a.n, line_docs, doc_state,
                                                none_counted, slot_cap);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int ddo = occupancy(mime_decode_docs_kernel<true>, 32 * kDocWarps, g_ddo_occ[di.device & 63]);
    e = launch_dependent(mime_decode_docs_kernel<true>, unsigned(di.sm_count * ddo), 32 * kDocWarps,
                         0, st, a.src, a.src_off, a.n, a.dst, a.dst_off, tabs, a.alph_id,
                         status_docs, line_docs, states, none_counted, slot_cap);
    if (e != cudaSuccess) return e;
    const int cd = occupancy(mime_count_docs_kernel, kCountThreads, g_cd_occ[di.device & 63]);
    e = launch_dependent(mime_count_docs_kernel, unsigned(di.sm_count * cd), kCountThreads, 0, st,
                         a.src, a.src_off, a.n, states, line_docs, none_counted, slot_cap);
    if (e != cudaSuccess) return e;
    e = launch_dependent(mime_scan_docs_kernel, sb, 256, 0, st, a.src, a.src_off, a.n, states,
                         doc_state, line_docs, status_docs, none_counted, slot_cap);
    if (e != cudaSuccess) return e;
    const int dd = occupancy(mime_decode_docs_kernel<false>, 32 * kDocWarps, g_dd_occ[di.device & 63]);
    e = launch_dependent(mime_decode_docs_kernel<false>, unsigned(di.sm_count * dd), 32 * kDocWarps,
                         0, st, a.src, a.src_off, a.n, a.dst, a.dst_off, tabs, a.alph_id,
                         status_docs, line_docs, states, none_counted, slot_cap);
    if (e != cudaSuccess) return e;
    return launch_dependent(mime_finalize_docs_kernel, unsigned((a.n + 255) / 256), 256, 0, st,
                            a.src, a.src_off, a.n, tabs, a.alph_id, status_docs, doc_state,
                            slot_cap, a.results);
}

uint32_t mime_fault_flag(bool clear) {
    uint32_t v = 0;
    cudaMemcpyFromSymbol(&v, g_fault, sizeof(v));
    if (clear && v) {
        const uint32_t z = 0;
        cudaMemcpyToSymbol(g_fault, &z, sizeof(z));
    }
    return v;
}

}  // namespace b64
