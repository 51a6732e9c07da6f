// MIME-style strict decode: CR, LF and space are skipped, everything else is
// decoded as by the single-buffer decoder (Sec. 2 and Sec. 3.2 of Mula &
// Lemire) on the characters that remain; error offsets are reported in the
// original input. The paper cites MIME only as motivation (Sec. 1); the
// whitespace removal and this single-pass design are this library's.
//
// One pass over the input with decoupled look-back:
//   - CTAs claim tiles of kTile raw bytes in arrival order from an atomic
//     counter (so every tile's predecessors are already running);
//   - each thread classifies its 32 bytes; a warp/block scan gives every data
//     character its index within the tile;
//   - the tile publishes its aggregate (data characters, last data byte),
//     walks back over its predecessors' published states until it meets an
//     inclusive prefix, and publishes its own inclusive prefix; the prefix
//     tells it the global index of its first data character and the last data
//     byte before it (so the group of four that straddles the tile start can
//     be finished here);
//   - the tile compacts its characters' 6-bit values in shared memory and
//     writes exactly the output bytes whose second character it holds, up to
//     its first '=' or bad byte;
//   - bad bytes and the first '=' are folded into status words with atomic
//     minima; a one-thread kernel then applies the padding and length rules
//     on the compacted stream and writes the result.
// Every wait on a predecessor is bounded; a tile that gives up publishes a
// "poisoned" state so its successors stop at once, and the result becomes
// B64_E_TIMEOUT.
#include <mutex>

#include "b64_internal.h"

namespace b64 {
namespace {

constexpr int kThreads = 256;
constexpr int kChunks = 4;                              // rounds of 32 bytes per thread
constexpr uint32_t kChunk = kThreads * 32;              // 8 KiB
constexpr uint32_t kTile = kChunk * kChunks;            // raw bytes per tile (32 KiB)
constexpr uint32_t kSpace = 0xC0u;                      // table class of CR, LF, space

// Tile state word: [flag:2][last data byte:8][data characters:54].
constexpr int kFlagShift = 62;
constexpr uint64_t kCountMask = (uint64_t(1) << 54) - 1;
constexpr uint64_t kFlagAggregate = 1, kFlagPrefix = 2, kFlagPoison = 3;

__device__ uint32_t g_fault;

__host__ __device__ __forceinline__ uint64_t make_state(uint64_t flag, uint32_t last,
                                                        uint64_t count) {
    return (flag << kFlagShift) | (uint64_t(last & 0xFFu) << 54) | (count & kCountMask);
}
__host__ __device__ __forceinline__ uint64_t st_flag(uint64_t s) { return s >> kFlagShift; }
__host__ __device__ __forceinline__ uint32_t st_last(uint64_t s) {
    return uint32_t(s >> 54) & 0xFFu;
}
__host__ __device__ __forceinline__ uint64_t st_count(uint64_t s) { return s & kCountMask; }

__device__ __forceinline__ uint64_t ld_relaxed(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(unsigned long long* p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"((unsigned long long)v)
                 : "memory");
}

// Four already-translated 6-bit values (one per byte, first in the low byte)
// -> their 24-bit value a<<18 | b<<12 | c<<6 | d. Each byte is masked to six
// bits first, so that a byte holding anything larger (a value past the end of
// the valid data: stale shared memory) cannot carry into the output bytes of
// the other values.
__device__ __forceinline__ uint32_t decode4_values(uint32_t w) {
    w &= 0x3F3F3F3Fu;
    const uint32_t a = w & 0xFFu, b = (w >> 8) & 0xFFu, c = (w >> 16) & 0xFFu, d = w >> 24;
    return ((a * 64u + b) * 64u + c) * 64u + d;
}

__host__ __device__ __forceinline__ uint64_t bytes_for(uint64_t j) {
    const uint64_t r = j & 3;
    return 3 * (j >> 2) + (r ? r - 1 : 0);
}

// Dynamic shared memory: raw[kTile] (the tile; later the output bytes) then
// vals[kTile + 32] (compacted values at (P & 3) + index).
constexpr size_t kDynSmem = 2 * size_t(kTile) + 32;

struct TileShared {
    uint8_t lut[256];                       // 0..63, 0x80 (bad or '='), kSpace
    unsigned long long warp_tot[kThreads / 32];
    unsigned long long tile;
    unsigned long long excl;
    uint32_t prev_last;
    uint32_t poisoned;
    uint32_t last_key;                      // (raw position + 1) << 8 | byte of the last data byte
    uint32_t min_bad_raw, min_eq_raw, min_eq_comp, min_stop_comp;
};

// The tile's predecessors' published states, 32 at a time (warp 0): the data
// characters before the tile and the last data byte before it. Returns false
// if a wait ran out or a predecessor was poisoned.
__device__ bool look_back(const unsigned long long* __restrict__ states, uint64_t tile,
                          const unsigned long long* timeout, uint64_t wait_limit_ns,
                          uint64_t* excl_out, uint32_t* prev_last_out, bool* have_prev_out) {
    const int lane = threadIdx.x & 31;
    uint64_t excl = 0;
    uint32_t prev_last = 0;
    bool have_prev = false;
    int64_t wend = int64_t(tile);
    const uint64_t t0 = global_timer_ns();
    for (;;) {
        const int64_t t = wend - 1 - lane;
        uint64_t s = t >= 0 ? ld_relaxed(states + t) : make_state(kFlagPrefix, 0, 0);
        uint32_t spins = 0;
        for (;;) {
            const bool ready = st_flag(s) != 0;
            if (__all_sync(0xffffffffu, ready)) break;
            if (!ready) s = ld_relaxed(states + t);
            if ((++spins & 31) == 0) {
                const bool give_up =
                    global_timer_ns() - t0 > wait_limit_ns || ld_relaxed(timeout) != 0;
                if (__any_sync(0xffffffffu, give_up)) return false;
            }
        }
        if (__any_sync(0xffffffffu, st_flag(s) == kFlagPoison)) return false;
        const uint32_t pmask = __ballot_sync(0xffffffffu, st_flag(s) == kFlagPrefix);
        const int pl = pmask ? __ffs(pmask) - 1 : 31;  // nearest inclusive prefix
        const bool mine = lane <= pl;
        uint64_t c = mine ? st_count(s) : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        excl += c;
        if (!have_prev) {
            const uint32_t lmask = __ballot_sync(0xffffffffu, mine && st_count(s) > 0);
            if (lmask) {
                prev_last = __shfl_sync(0xffffffffu, st_last(s), __ffs(lmask) - 1);
                have_prev = true;
            }
        }
        if (pmask) break;
        wend -= 32;
    }
    *excl_out = excl;
    *prev_last_out = prev_last;
    *have_prev_out = have_prev;
    return true;
}

__global__ void __launch_bounds__(kThreads, 2)
    mime_decode_kernel(const uint8_t* __restrict__ src, uint64_t m, uint8_t* __restrict__ dst,
                       const __grid_constant__ DecodeTable tab, int padded,
                       unsigned long long* __restrict__ status,
                       unsigned long long* __restrict__ states, uint64_t ntiles,
                       uint64_t skip_tiles, uint64_t wait_limit_ns) {
    __shared__ TileShared sh;
    extern __shared__ __align__(16) uint8_t dyn[];
    uint8_t* raw = dyn;
    uint8_t* vals = dyn + kTile;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < 64) reinterpret_cast<uint32_t*>(sh.lut)[tid] = tab.w[tid];
    __syncthreads();
    if (tid == 0) sh.lut['\r'] = sh.lut['\n'] = sh.lut[' '] = uint8_t(kSpace);
    const bool aligned = (reinterpret_cast<uintptr_t>(src) & 15u) == 0;
    unsigned long long* counter = status + 3;
    unsigned long long* timeout = status + 4;

    for (;;) {
        __syncthreads();  // every thread is done with the previous tile's shared state
        if (tid == 0) {
            sh.tile = atomicAdd(counter, 1ull) + skip_tiles;
            sh.min_bad_raw = sh.min_eq_raw = sh.min_eq_comp = sh.min_stop_comp = 0xFFFFFFFFu;
            sh.last_key = 0;
            sh.poisoned = 0;
        }
        __syncthreads();
        const uint64_t tile = sh.tile;
        if (tile >= ntiles) break;
        const uint64_t base = tile * kTile;
        const uint32_t len = uint32_t(m - base < kTile ? m - base : kTile);

        // ---- stage the tile (coalesced 16-byte loads; bytes past the end read as spaces)
#pragma unroll 1
        for (int half = 0; half < 2; ++half) {
            constexpr int kLoads = int(kTile / 16 / kThreads) / 2;
            uint4 v[kLoads];
#pragma unroll
            for (int i = 0; i < kLoads; ++i) {
                const uint32_t off = 16 * (tid + kThreads * (i + kLoads * half));
                if (aligned && off + 16 <= len) {
                    v[i] = *reinterpret_cast<const uint4*>(src + base + off);
                } else {
                    uint8_t* b = reinterpret_cast<uint8_t*>(&v[i]);
                    for (int k = 0; k < 16; ++k) b[k] = off + k < len ? src[base + off + k] : 32;
                }
            }
#pragma unroll
            for (int i = 0; i < kLoads; ++i)
                *reinterpret_cast<uint4*>(raw + 16 * (tid + kThreads * (i + kLoads * half))) =
                    v[i];
        }
        __syncthreads();

        // ---- count data characters per 32-byte piece; 4 pieces per thread,
        //      piece c covers raw bytes [c*kChunk + 32*tid, +32)
        uint64_t cnt = 0;  // four 16-bit counts, piece c in bits 16c..16c+15
        uint32_t my_last = 0;
#pragma unroll 1
        for (int c = 0; c < kChunks; ++c) {
            const uint32_t p0 = c * kChunk + 32 * tid;
            const uint4 x = *reinterpret_cast<const uint4*>(raw + p0);
            const uint4 y = *reinterpret_cast<const uint4*>(raw + p0 + 16);
            const uint32_t w[8] = {x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w};
            uint32_t k = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q)
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const uint32_t ch = __byte_perm(w[q], 0, 0x4440u + i);
                    if (sh.lut[ch] != kSpace) {
                        ++k;
                        my_last = ((p0 + 4 * q + i + 1) << 8) | ch;  // never 0
                    }
                }
            cnt |= uint64_t(k) << (16 * c);
        }
        if (my_last) atomicMax(&sh.last_key, my_last);
        uint64_t incl = cnt;  // scan of the four counts at once (fields never overflow)
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) sh.warp_tot[warp] = incl;
        __syncthreads();
        uint64_t before = 0, total = 0;
#pragma unroll
        for (int q = 0; q < kThreads / 32; ++q) {
            if (q < warp) before += sh.warp_tot[q];
            total += sh.warp_tot[q];
        }
        const uint64_t excl_fields = before + incl - cnt;
        // piece c of this thread starts at data index
        //   (totals of pieces < c) + (this thread's exclusive count in piece c)
        uint32_t tile_count = 0;
#pragma unroll
        for (int c = 0; c < kChunks; ++c) tile_count += uint32_t((total >> (16 * c)) & 0xFFFFu);
        const uint32_t tile_last = sh.last_key & 0xFFu;
        const bool tile_has_last = sh.last_key != 0;

        // ---- publish the aggregate, look back, publish the inclusive prefix
        if (warp == 0) {
            unsigned long long* my = states + tile;
            uint64_t excl = 0;
            uint32_t prev_last = 0;
            bool have_prev = false, ok = true;
            if (tile == 0) {
                if (lane == 0) st_relaxed(my, make_state(kFlagPrefix, tile_last, tile_count));
            } else {
                if (lane == 0) st_relaxed(my, make_state(kFlagAggregate, tile_last, tile_count));
                ok = look_back(states, tile, timeout, wait_limit_ns, &excl, &prev_last,
                               &have_prev);
                if (lane == 0) {
                    if (ok) {
                        st_relaxed(my, make_state(kFlagPrefix,
                                                  tile_has_last ? tile_last : prev_last,
                                                  excl + tile_count));
                    } else {
                        st_relaxed(my, make_state(kFlagPoison, 0, 0));
                        atomicExch(timeout, 1ull);
                        atomicOr(&g_fault, 1u);
                    }
                }
            }
            if (lane == 0) {
                sh.excl = excl;
                sh.prev_last = have_prev ? prev_last : 0u;
                sh.poisoned = ok ? 0u : 1u;
            }
        }
        __syncthreads();
        if (sh.poisoned) continue;  // uniform: the whole block skips this tile
        const uint64_t P = sh.excl;
        const uint32_t shift = uint32_t(P & 3);

        // ---- compact the 6-bit values to vals[shift + index]; note errors
        if (tid == 0 && shift) vals[shift - 1] = sh.lut[sh.prev_last];
        uint32_t bad_raw = 0xFFFFFFFFu, eq_raw = 0xFFFFFFFFu, eq_comp = 0xFFFFFFFFu,
                 stop = 0xFFFFFFFFu;
#pragma unroll 1
        for (int c = 0; c < kChunks; ++c) {
            const uint32_t p0 = c * kChunk + 32 * tid;
            uint32_t pos = uint32_t((excl_fields >> (16 * c)) & 0xFFFFu);
            for (int c2 = 0; c2 < c; ++c2) pos += uint32_t((total >> (16 * c2)) & 0xFFFFu);
            const uint4 x = *reinterpret_cast<const uint4*>(raw + p0);
            const uint4 y = *reinterpret_cast<const uint4*>(raw + p0 + 16);
            const uint32_t w[8] = {x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w};
#pragma unroll
            for (int q = 0; q < 8; ++q)
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const uint32_t ch = __byte_perm(w[q], 0, 0x4440u + i);
                    const uint32_t v = sh.lut[ch];
                    if (v != kSpace) {
                        vals[shift + pos] = uint8_t(v);
                        if (v & kBad) {
                            if (stop == 0xFFFFFFFFu) stop = pos;
                            const uint32_t raw = p0 + 4 * q + i;
                            if (ch == '=' && padded) {
                                if (eq_raw == 0xFFFFFFFFu) {
                                    eq_raw = raw;
                                    eq_comp = pos;
                                }
                            } else if (bad_raw == 0xFFFFFFFFu) {
                                bad_raw = raw;
                            }
                        }
                        ++pos;
                    }
                }
        }
        if (stop != 0xFFFFFFFFu) {
            atomicMin(&sh.min_stop_comp, stop);
            if (bad_raw != 0xFFFFFFFFu) atomicMin(&sh.min_bad_raw, bad_raw);
            if (eq_raw != 0xFFFFFFFFu) {
                atomicMin(&sh.min_eq_raw, eq_raw);
                atomicMin(&sh.min_eq_comp, eq_comp);
            }
        }
        __syncthreads();
        if (tid == 0) {
            if (sh.min_bad_raw != 0xFFFFFFFFu) atomicMin(status + 0, base + sh.min_bad_raw);
            if (sh.min_eq_raw != 0xFFFFFFFFu) {
                atomicMin(status + 1, base + sh.min_eq_raw);
                atomicMin(status + 2, P + sh.min_eq_comp);
            }
        }

        // ---- whole quads, four per thread: 16 values -> 12 bytes into the raw
        //      buffer (free now); quad Q's values sit at vals[4 * (Q - P/4)]
        const uint32_t jend = sh.min_stop_comp < tile_count ? sh.min_stop_comp : tile_count;
        const uint64_t ob = bytes_for(P), oe = bytes_for(P + jend);
        const uint32_t nout = uint32_t(oe > ob ? oe - ob : 0);
        const uint32_t skip = shift ? shift - 1 : 0;    // bytes of the first quad not ours
        const uint32_t ngroups = (shift + jend + 15) / 16;
        uint8_t* out = raw;
        for (uint32_t g = tid; g < ngroups; g += kThreads) {
            const uint4 c = *reinterpret_cast<const uint4*>(vals + 16 * g);
            const uint3 o = pack4x24(decode4_values(c.x), decode4_values(c.y),
                                     decode4_values(c.z), decode4_values(c.w));
            uint32_t* ow = reinterpret_cast<uint32_t*>(out + 12 * g);
            ow[0] = o.x;
            ow[1] = o.y;
            ow[2] = o.z;
        }
        __syncthreads();
        // copy out: aligned 16-byte stores for the middle, bytes at the edges
        uint8_t* q = dst + ob;
        const uint32_t head = uint32_t((16 - (reinterpret_cast<uintptr_t>(q) & 15)) & 15);
        const uint32_t h = head < nout ? head : nout;
        if (tid < int(h)) q[tid] = out[skip + tid];
        const uint32_t body = (nout - h) & ~15u;
        for (uint32_t k = tid; k < body / 16; k += kThreads) {
            const uint32_t off = skip + h + 16 * k;
            *reinterpret_cast<uint4*>(q + h + 16 * k) = load16_shifted(out, off, off & 3);
        }
        for (uint32_t i = h + body + tid; i < nout; i += kThreads) q[i] = out[skip + i];
    }
}

// One thread: the padding and length rules on the compacted stream.
__global__ void mime_finalize_kernel(uint64_t m, int padded,
                                     const unsigned long long* __restrict__ status,
                                     const unsigned long long* __restrict__ states,
                                     uint64_t ntiles, int64_t* __restrict__ d_result) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (status[4]) {
        *d_result = B64_E_TIMEOUT;
        return;
    }
    const uint64_t last_state = ntiles ? states[ntiles - 1] : make_state(kFlagPrefix, 0, 0);
    const uint64_t mc = st_count(last_state);           // data characters
    const uint32_t last = st_last(last_state);
    uint64_t err = status[0];
    uint64_t pads = 0;
    if (padded && status[2] != kNoError) {
        const uint64_t qe = status[2];
        const bool ok = qe + 1 == mc || (qe + 2 == mc && last == '=');
        if (ok) pads = mc - qe;
        else err = status[1] < err ? status[1] : err;
    }
    if (padded ? (mc % 4 != 0) : (mc % 4 == 1)) err = m < err ? m : err;
    *d_result = err != kNoError ? -int64_t(err) - 1 : int64_t(bytes_for(mc - pads));
}

struct Occ {
    std::once_flag once;
    cudaError_t err = cudaSuccess;
    int ctas = 1;
};
Occ g_occ[64];

}  // namespace

size_t mime_workspace_bytes(uint64_t m) {
    const uint64_t ntiles = (m + kTile - 1) / kTile;
    return 64 + 8 * size_t(ntiles);
}

cudaError_t launch_mime_decode(const uint8_t* src, uint64_t m, uint8_t* dst,
                               const DecodeTable& tab, int padded, int64_t* d_result,
                               void* workspace, uint64_t skip_tiles, uint64_t wait_limit_ns,
                               cudaStream_t st) {
    const uint64_t ntiles = (m + kTile - 1) / kTile;
    unsigned long long* status = static_cast<unsigned long long*>(workspace);
    unsigned long long* states = status + 8;
    // status[0..2] (first bad byte, first '=' raw and compacted) start at "none";
    // the tile counter, the timeout word and every tile state start at zero.
    cudaError_t e = cudaMemsetAsync(status, 0xFF, 3 * sizeof(uint64_t), st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(status + 3, 0, (5 + ntiles) * sizeof(uint64_t), st);
    if (e != cudaSuccess) return e;
    if (ntiles) {
        const DeviceInfo& di = device_info();
        Occ& occ = g_occ[di.device & 63];
        std::call_once(occ.once, [&] {
            int c = 1;
            occ.err = cudaFuncSetAttribute(mime_decode_kernel,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           int(kDynSmem));
            if (occ.err == cudaSuccess &&
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, mime_decode_kernel, kThreads,
                                                              kDynSmem) != cudaSuccess)
                c = 1;
            occ.ctas = c > 0 ? c : 1;
        });
        if (occ.err != cudaSuccess) return occ.err;
        uint64_t grid = uint64_t(di.sm_count) * occ.ctas;
        if (ntiles < grid) grid = ntiles;
        mime_decode_kernel<<<unsigned(grid), kThreads, kDynSmem, st>>>(
            src, m, dst, tab, padded, status, states, ntiles, skip_tiles, wait_limit_ns);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    mime_finalize_kernel<<<1, 32, 0, st>>>(m, padded, status, states, ntiles, d_result);
    return cudaGetLastError();
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
