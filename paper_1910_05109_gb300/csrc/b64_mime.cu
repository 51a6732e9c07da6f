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
constexpr int kPerThread = 32;
constexpr uint32_t kTile = kThreads * kPerThread;       // raw bytes per tile
constexpr uint32_t kOutCap = kTile / 4 * 3 + 32;        // output bytes a tile may write

// Tile state word: [flag:2][last data byte:8][data characters:54].
constexpr int kFlagShift = 62;
constexpr uint64_t kCountMask = (uint64_t(1) << 54) - 1;
constexpr uint64_t kFlagAggregate = 1, kFlagPrefix = 2, kFlagPoison = 3;

__device__ uint32_t g_fault;

__device__ __forceinline__ uint64_t make_state(uint64_t flag, uint32_t last, uint64_t count) {
    return (flag << kFlagShift) | (uint64_t(last & 0xFFu) << 54) | (count & kCountMask);
}
__device__ __forceinline__ uint64_t st_flag(uint64_t s) { return s >> kFlagShift; }
__device__ __forceinline__ uint32_t st_last(uint64_t s) { return uint32_t(s >> 54) & 0xFFu; }
__device__ __forceinline__ uint64_t st_count(uint64_t s) { return s & kCountMask; }

__device__ __forceinline__ uint64_t ld_relaxed(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(unsigned long long* p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"((unsigned long long)v)
                 : "memory");
}

__host__ __device__ __forceinline__ uint64_t bytes_for(uint64_t j) {
    const uint64_t r = j & 3;
    return 3 * (j >> 2) + (r ? r - 1 : 0);
}

__device__ __forceinline__ bool is_space(uint32_t c) { return c == 13 || c == 10 || c == 32; }

struct TileShared {
    uint8_t lut[256];
    uint8_t vals[kTile];
    uint8_t out[kOutCap + 16];
    uint32_t warp_count[kThreads / 32];
    uint32_t warp_last[kThreads / 32];
    unsigned long long tile;
    unsigned long long excl;
    uint32_t prev_last;
    uint32_t poisoned;
    uint32_t min_bad_raw, min_eq_raw, min_eq_comp, min_stop_comp;
};

__global__ void __launch_bounds__(kThreads)
    mime_decode_kernel(const uint8_t* __restrict__ src, uint64_t m, uint8_t* __restrict__ dst,
                       const __grid_constant__ DecodeTable tab, int padded,
                       unsigned long long* __restrict__ status,
                       unsigned long long* __restrict__ states, uint64_t ntiles,
                       uint64_t skip_tiles, uint64_t wait_limit_ns) {
    __shared__ __align__(16) TileShared sh;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < 64) reinterpret_cast<uint32_t*>(sh.lut)[tid] = tab.w[tid];
    const bool aligned = (reinterpret_cast<uintptr_t>(src) & 15u) == 0;
    unsigned long long* counter = status + 3;
    unsigned long long* timeout = status + 4;

    for (;;) {
        __syncthreads();  // every thread is done with the previous tile's shared state
        if (tid == 0) {
            sh.tile = atomicAdd(counter, 1ull) + skip_tiles;
            sh.min_bad_raw = sh.min_eq_raw = sh.min_eq_comp = sh.min_stop_comp = 0xFFFFFFFFu;
            sh.poisoned = 0;
        }
        __syncthreads();
        const uint64_t tile = sh.tile;
        if (tile >= ntiles) break;
        const uint64_t base = tile * kTile;
        const uint32_t len = uint32_t(m - base < kTile ? m - base : kTile);

        // ---- load and classify this thread's 32 bytes (absent bytes read as spaces)
        uint32_t w[8];
        const uint32_t lo = uint32_t(tid) * kPerThread;
        if (aligned && lo + kPerThread <= len) {
            const uint4 a = *reinterpret_cast<const uint4*>(src + base + lo);
            const uint4 b = *reinterpret_cast<const uint4*>(src + base + lo + 16);
            w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
            w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                uint32_t v = 0;
                for (int i = 0; i < 4; ++i) {
                    const uint32_t p = lo + 4 * k + i;
                    v |= uint32_t(p < len ? src[base + p] : 32u) << (8 * i);
                }
                w[k] = v;
            }
        }
        uint32_t count = 0, last = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const uint32_t c = (w[k] >> (8 * i)) & 0xFFu;
                if (!is_space(c)) {
                    ++count;
                    last = c;
                }
            }

        // ---- block scan of data-character counts; the tile's last data byte
        uint32_t incl = count;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const uint32_t nonempty = __ballot_sync(0xffffffffu, count > 0);
        const uint32_t wlast =
            __shfl_sync(0xffffffffu, last, nonempty ? 31 - __clz(nonempty) : 0);
        if (lane == 31) {
            sh.warp_count[warp] = incl;
            sh.warp_last[warp] = nonempty ? (wlast | 0x100u) : 0u;
        }
        __syncthreads();
        uint32_t wbase = 0, tile_count = 0, tile_last = 0;
        bool tile_has_last = false;
        for (int q = 0; q < kThreads / 32; ++q) {
            if (q < warp) wbase += sh.warp_count[q];
            tile_count += sh.warp_count[q];
            if (sh.warp_last[q]) {
                tile_last = sh.warp_last[q] & 0xFFu;
                tile_has_last = true;
            }
        }
        const uint32_t excl_local = wbase + incl - count;

        // ---- publish, look back, publish the inclusive prefix
        if (tid == 0) {
            unsigned long long* my = states + tile;
            uint64_t excl = 0;
            uint32_t prev_last = 0;
            bool have_prev = false, poison = false;
            if (tile == 0) {
                st_relaxed(my, make_state(kFlagPrefix, tile_last, tile_count));
            } else {
                st_relaxed(my, make_state(kFlagAggregate, tile_last, tile_count));
                const uint64_t t0 = global_timer_ns();
                for (int64_t t = int64_t(tile) - 1; t >= 0; --t) {
                    uint64_t s = ld_relaxed(states + t);
                    uint32_t spins = 0;
                    while (st_flag(s) == 0) {
                        // give up after the limit, or as soon as any tile has given up
                        if ((++spins & 63) == 0 &&
                            (global_timer_ns() - t0 > wait_limit_ns || ld_relaxed(timeout)))
                            break;
                        s = ld_relaxed(states + t);
                    }
                    const uint64_t f = st_flag(s);
                    if (f == 0 || f == kFlagPoison) {
                        poison = true;
                        break;
                    }
                    if (!have_prev && st_count(s) > 0) {
                        prev_last = st_last(s);
                        have_prev = true;
                    }
                    excl += st_count(s);
                    if (f == kFlagPrefix) break;
                }
                if (poison) {
                    st_relaxed(my, make_state(kFlagPoison, 0, 0));
                    atomicExch(timeout, 1ull);
                    atomicOr(&g_fault, 1u);
                } else {
                    st_relaxed(my, make_state(kFlagPrefix, tile_has_last ? tile_last : prev_last,
                                              excl + tile_count));
                }
            }
            sh.excl = excl;
            sh.prev_last = have_prev ? prev_last : 0u;
            sh.poisoned = poison ? 1u : 0u;
        }
        __syncthreads();
        if (sh.poisoned) continue;  // uniform: the whole block skips this tile
        const uint64_t P = sh.excl;

        // ---- compact the 6-bit values; note the first bad byte and first '='
        uint32_t pos = excl_local;
        uint32_t bad_raw = 0xFFFFFFFFu, eq_raw = 0xFFFFFFFFu, eq_comp = 0xFFFFFFFFu,
                 stop = 0xFFFFFFFFu;
#pragma unroll
        for (int k = 0; k < 8; ++k)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const uint32_t c = (w[k] >> (8 * i)) & 0xFFu;
                if (!is_space(c)) {
                    const uint32_t v = sh.lut[c];
                    sh.vals[pos] = uint8_t(v);
                    if (v & kBad) {
                        if (stop == 0xFFFFFFFFu) stop = pos;
                        const uint32_t raw = lo + 4 * k + i;
                        if (c == '=' && padded) {
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

        // ---- the output bytes whose second character is here, before any '=' / bad byte
        const uint32_t jend = sh.min_stop_comp < tile_count ? sh.min_stop_comp : tile_count;
        const uint64_t ob = bytes_for(P), oe = bytes_for(P + jend);
        const uint32_t nout = uint32_t(oe > ob ? oe - ob : 0);
        const uint32_t vprev = sh.lut[sh.prev_last];
        for (uint32_t t = tid; t < nout; t += kThreads) {
            const uint64_t b = ob + t;
            const uint64_t q = b / 3;
            const uint32_t r = uint32_t(b - 3 * q);
            const uint64_t j = 4 * q + r + 1;  // global index of the pair's second character
            const uint32_t jl = uint32_t(j - P);
            const uint32_t v1 = jl >= 1 ? sh.vals[jl - 1] : vprev;
            const uint32_t v2 = sh.vals[jl];
            uint32_t byte;
            if (r == 0) byte = (v1 << 2) | (v2 >> 4);
            else if (r == 1) byte = ((v1 & 15u) << 4) | (v2 >> 2);
            else byte = ((v1 & 3u) << 6) | v2;
            sh.out[t] = uint8_t(byte);
        }
        __syncthreads();
        // copy out: aligned 16-byte stores for the middle, bytes at the edges
        uint8_t* q = dst + ob;
        const uint32_t head = uint32_t((16 - (reinterpret_cast<uintptr_t>(q) & 15)) & 15);
        const uint32_t h = head < nout ? head : nout;
        if (tid < int(h)) q[tid] = sh.out[tid];
        const uint32_t body = (nout - h) & ~15u;
        for (uint32_t k = tid; k < body / 16; k += kThreads) {
            const uint32_t off = h + 16 * k;
            *reinterpret_cast<uint4*>(q + off) = load16_shifted(sh.out, off, off & 3);
        }
        for (uint32_t i = h + body + tid; i < nout; i += kThreads) q[i] = sh.out[i];
        __syncthreads();
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
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, mime_decode_kernel, kThreads,
                                                              0) != cudaSuccess)
                c = 1;
            occ.ctas = c > 0 ? c : 1;
        });
        uint64_t grid = uint64_t(di.sm_count) * occ.ctas;
        if (ntiles < grid) grid = ntiles;
        mime_decode_kernel<<<unsigned(grid), kThreads, 0, st>>>(
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
