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
//   1. prep kernel (one block): tiles per string, exclusive scan into the
//      caller's workspace; encode writes each string's output length to
//      results, decode sets each string's error word to "none";
//   2. tile kernel (persistent): every warp takes an equal, contiguous range
//      of tiles, finds the string of its first tile by binary search over the
//      scan and then walks forward. A tile is staged through the warp's
//      shared memory with aligned 16-byte loads (strings start anywhere),
//      re-aligned with funnel shifts, coded with the same per-unit steps as
//      the single-buffer kernels, and copied out with aligned 16-byte stores
//      and byte stores at the edges. Decode tiles fold bad-byte offsets into
//      the string's error word with an atomic minimum;
//   3. decode only: one thread per string applies the padding and length
//      rules to the string's last 2..5 characters and writes its result.
#include <mutex>

#include "b64_internal.h"

namespace b64 {
namespace {

constexpr int kPrepThreads = 1024;

// Warps per block of the tile kernels: the per-warp staging buffers are
// static shared memory, which must stay under 48 KiB per block.
template <int U>
struct TileShape {
    static constexpr int kWarps = U >= 8 ? 4 : 8;
    static constexpr int kThreads = 32 * kWarps;
};

__host__ __device__ __forceinline__ uint64_t dec_body_length(uint64_t m) {
    return m >= 2 ? ((m - 2) & ~uint64_t(3)) : 0;
}

__host__ __device__ __forceinline__ uint64_t enc_length(uint64_t n, int padded) {
    const uint64_t g = n / 3, r = n % 3;
    return r == 0 ? 4 * g : 4 * g + (padded ? 4 : r + 1);
}

// ------------------------------------------------------------------ prep
// tile_start[0..n] = exclusive scan of tiles per string (tile_start[n] = total).
template <bool kDecode>
__global__ void __launch_bounds__(kPrepThreads)
    batch_prep_kernel(const int64_t* __restrict__ src_off, int64_t n, uint32_t tile_bytes,
                      const __grid_constant__ BatchTables tabs, const uint8_t* __restrict__ alph_id,
                      int64_t* __restrict__ tile_start, int64_t* __restrict__ results,
                      unsigned long long* __restrict__ err) {
    __shared__ int64_t part[kPrepThreads];
    const int tid = threadIdx.x;
    const int64_t per = (n + kPrepThreads - 1) / kPrepThreads;
    const int64_t b = per * tid, e = b + per < n ? b + per : n;
    int64_t sum = 0;
    for (int64_t i = b; i < e; ++i) {
        const uint64_t len = uint64_t(src_off[i + 1] - src_off[i]);
        const uint64_t work = kDecode ? dec_body_length(len) : len;
        sum += int64_t((work + tile_bytes - 1) / tile_bytes);
    }
    part[tid] = sum;
    __syncthreads();
    for (int o = 1; o < kPrepThreads; o <<= 1) {  // inclusive scan of the partial sums
        const int64_t v = tid >= o ? part[tid - o] : 0;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    int64_t run = part[tid] - sum;
    for (int64_t i = b; i < e; ++i) {
        tile_start[i] = run;
        const uint64_t len = uint64_t(src_off[i + 1] - src_off[i]);
        const uint64_t work = kDecode ? dec_body_length(len) : len;
        run += int64_t((work + tile_bytes - 1) / tile_bytes);
        if (kDecode) {
            err[i] = kNoError;
        } else {
            const int a = alph_id ? (alph_id[i] & (kMaxAlphabets - 1)) : 0;
            results[i] = int64_t(enc_length(len, tabs.padded[a]));
        }
    }
    if (tid == kPrepThreads - 1) tile_start[n] = part[kPrepThreads - 1];
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

// Writes sbuf[0 .. len) to global q (any alignment): aligned 16-byte stores
// for the middle, byte stores for the ragged head and tail. Warp-collective.
__device__ __forceinline__ void warp_stage_out(uint8_t* q, const uint8_t* sbuf, uint32_t len,
                                               int lane) {
    const uint32_t head = uint32_t((16 - (reinterpret_cast<uintptr_t>(q) & 15)) & 15);
    const uint32_t h = head < len ? head : len;
    if (lane < int(h)) q[lane] = sbuf[lane];
    const uint32_t body = (len - h) & ~15u;
    const uint32_t sh = h & 3;
    for (uint32_t k = lane; k < body / 16; k += 32) {
        const uint32_t off = h + 16 * k;
        *reinterpret_cast<uint4*>(q + off) = load16_shifted(sbuf, off, sh);
    }
    for (uint32_t i = h + body + lane; i < len; i += 32) q[i] = sbuf[i];
}

// Binary search (every lane computes the same result): the string s with
// tile_start[s] <= t < tile_start[s+1], which skips strings with no tiles.
__device__ __forceinline__ int64_t find_string(const int64_t* __restrict__ tile_start, int64_t n,
                                               int64_t t) {
    int64_t lo = 0, hi = n;  // invariant: tile_start[lo] <= t < tile_start[hi]
    while (hi - lo > 1) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (tile_start[mid] <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

// ------------------------------------------------------------------ encode tiles
template <int U>
__global__ void __launch_bounds__(TileShape<U>::kThreads)
    encode_batch_kernel(const uint8_t* __restrict__ src, const int64_t* __restrict__ src_off,
                        int64_t n, uint8_t* __restrict__ dst, const int64_t* __restrict__ dst_off,
                        const __grid_constant__ BatchTables tabs,
                        const uint8_t* __restrict__ alph_id,
                        const int64_t* __restrict__ tile_start) {
    constexpr int kWarps = TileShape<U>::kWarps, kThreads = TileShape<U>::kThreads;
    constexpr uint32_t T = 32 * U * 12;        // input bytes per tile
    constexpr uint32_t TO = T / 3 * 4 + 4;     // output characters per tile (+ padding group)
    constexpr uint32_t SIN = T + 32;           // staging room for a ragged start
    constexpr uint32_t SOUT = (TO + 16 + 15) & ~15u;  // rows stay 16-byte aligned
    __shared__ __align__(16) uint8_t luts[kMaxAlphabets][64];
    __shared__ __align__(16) uint8_t sin_all[kWarps][SIN];
    __shared__ __align__(16) uint8_t sout_all[kWarps][SOUT];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < kMaxAlphabets * 16; i += kThreads)
        reinterpret_cast<uint32_t*>(luts)[i] = tabs.enc[i / 16].w[i % 16];
    __syncthreads();
    uint8_t* sin = sin_all[warp];
    uint8_t* sout = sout_all[warp];

    const int64_t total = tile_start[n];
    const int64_t GW = int64_t(gridDim.x) * kWarps;
    const int64_t gw = int64_t(blockIdx.x) * kWarps + warp;
    const int64_t per = (total + GW - 1) / GW;
    const int64_t t0 = gw * per, t1 = t0 + per < total ? t0 + per : total;
    if (t0 >= t1) return;
    int64_t s = find_string(tile_start, n, t0);
    const uint64_t src_end = uint64_t(src_off[n]);

    for (int64_t t = t0; t < t1; ++t) {
        while (t >= tile_start[s + 1]) ++s;
        const int64_t lt = t - tile_start[s];
        const uint64_t s0 = uint64_t(src_off[s]), s1 = uint64_t(src_off[s + 1]);
        const uint64_t a = s0 + uint64_t(lt) * T;
        const uint64_t b = a + T < s1 ? a + T : s1;
        const bool last = b == s1;
        const int ai = alph_id ? (alph_id[s] & (kMaxAlphabets - 1)) : 0;
        const uint8_t* lut = luts[ai];
        const uint32_t nbytes = uint32_t(b - a);
        const uint32_t triples = nbytes / 3;
        const uint32_t delta = uint32_t((reinterpret_cast<uintptr_t>(src + a)) & 15);

        __syncwarp();
        warp_stage_in(sin, src, a, b, 0, src_end, lane);
        __syncwarp();
        const uint32_t sh = delta & 3;
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
        warp_stage_out(dst + dst_off[s] + uint64_t(lt) * (T / 3 * 4), sout, nout, lane);
    }
}

// ------------------------------------------------------------------ decode tiles
template <int U>
__global__ void __launch_bounds__(TileShape<U>::kThreads)
    decode_batch_kernel(const uint8_t* __restrict__ src, const int64_t* __restrict__ src_off,
                        int64_t n, uint8_t* __restrict__ dst, const int64_t* __restrict__ dst_off,
                        const __grid_constant__ BatchTables tabs,
                        const uint8_t* __restrict__ alph_id,
                        const int64_t* __restrict__ tile_start,
                        unsigned long long* __restrict__ err) {
    constexpr int kWarps = TileShape<U>::kWarps, kThreads = TileShape<U>::kThreads;
    constexpr uint32_t T = 32 * U * 16;  // characters per tile
    constexpr uint32_t TO = T / 4 * 3;   // output bytes per tile
    constexpr uint32_t SIN = T + 32;
    constexpr uint32_t SOUT = (TO + 16 + 15) & ~15u;
    __shared__ __align__(16) uint8_t luts[kMaxAlphabets][256];
    __shared__ __align__(16) uint8_t sin_all[kWarps][SIN];
    __shared__ __align__(16) uint8_t sout_all[kWarps][SOUT];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < kMaxAlphabets * 64; i += kThreads)
        reinterpret_cast<uint32_t*>(luts)[i] = tabs.dec[i / 64].w[i % 64];
    __syncthreads();
    uint8_t* sin = sin_all[warp];
    uint8_t* sout = sout_all[warp];

    const int64_t total = tile_start[n];
    const int64_t GW = int64_t(gridDim.x) * kWarps;
    const int64_t gw = int64_t(blockIdx.x) * kWarps + warp;
    const int64_t per = (total + GW - 1) / GW;
    const int64_t t0 = gw * per, t1 = t0 + per < total ? t0 + per : total;
    if (t0 >= t1) return;
    int64_t s = find_string(tile_start, n, t0);
    const uint64_t src_end = uint64_t(src_off[n]);

    for (int64_t t = t0; t < t1; ++t) {
        while (t >= tile_start[s + 1]) ++s;
        const int64_t lt = t - tile_start[s];
        const uint64_t s0 = uint64_t(src_off[s]);
        const uint64_t body = dec_body_length(uint64_t(src_off[s + 1]) - s0);
        const uint64_t a = s0 + uint64_t(lt) * T;
        const uint64_t b = a + T < s0 + body ? a + T : s0 + body;
        const uint8_t* lut = luts[alph_id ? (alph_id[s] & (kMaxAlphabets - 1)) : 0];
        const uint32_t nchars = uint32_t(b - a);  // a multiple of 4
        const uint32_t delta = uint32_t((reinterpret_cast<uintptr_t>(src + a)) & 15);

        __syncwarp();
        warp_stage_in(sin, src, a, b, 0, src_end, lane);
        __syncwarp();
        const uint32_t sh = delta & 3;
        uint64_t first = kNoError;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t j = lane + 32 * u;
            if (16 * j + 16 <= nchars) {
                const uint4 c = load16_shifted(sin, delta + 16 * j, sh);
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
                            const uint64_t off = uint64_t(lt) * T + 16 * j + i;
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
                                const uint64_t off = uint64_t(lt) * T + 4 * q + i;
                                first = off < first ? off : first;
                                break;
                            }
                        }
                    }
                }
            }
        }
        const uint64_t wmin = warp_min_u64(first);
        if (lane == 0 && wmin != kNoError) atomicMin(&err[s], (unsigned long long)wmin);
        __syncwarp();
        warp_stage_out(dst + dst_off[s] + uint64_t(lt) * TO, sout, nchars / 4 * 3, lane);
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
    if (e != kNoError) {
        results[i] = -int64_t(e) - 1;
        return;
    }
    const uint32_t d = tail - pads;
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
    int ctas = 1;
};

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

Occ g_enc_occ[4][64], g_dec_occ[4][64];

int unit_slot(int units) { return units == 1 ? 0 : units == 2 ? 1 : units == 4 ? 2 : 3; }

template <int U>
cudaError_t launch_encode_tiles(const BatchArgs& a, const BatchTables& t, const int64_t* tiles,
                                cudaStream_t st) {
    const DeviceInfo& di = device_info();
    constexpr int threads = TileShape<U>::kThreads;
    const int occ =
        occupancy(encode_batch_kernel<U>, threads, g_enc_occ[unit_slot(U)][di.device & 63]);
    encode_batch_kernel<U><<<unsigned(di.sm_count * occ), threads, 0, st>>>(
        a.src, a.src_off, a.n, a.dst, a.dst_off, t, a.alph_id, tiles);
    return cudaGetLastError();
}

template <int U>
cudaError_t launch_decode_tiles(const BatchArgs& a, const BatchTables& t, const int64_t* tiles,
                                unsigned long long* err, cudaStream_t st) {
    const DeviceInfo& di = device_info();
    constexpr int threads = TileShape<U>::kThreads;
    const int occ =
        occupancy(decode_batch_kernel<U>, threads, g_dec_occ[unit_slot(U)][di.device & 63]);
    decode_batch_kernel<U><<<unsigned(di.sm_count * occ), threads, 0, st>>>(
        a.src, a.src_off, a.n, a.dst, a.dst_off, t, a.alph_id, tiles, err);
    return cudaGetLastError();
}

// dst_off = exclusive scan of per-string output capacities (one block).
template <bool kDecode>
__global__ void __launch_bounds__(kPrepThreads)
    batch_offsets_kernel(const int64_t* __restrict__ src_off, int64_t n,
                         const __grid_constant__ BatchTables tabs,
                         const uint8_t* __restrict__ alph_id, int64_t* __restrict__ dst_off) {
    __shared__ int64_t part[kPrepThreads];
    const int tid = threadIdx.x;
    const int64_t per = (n + kPrepThreads - 1) / kPrepThreads;
    const int64_t b = per * tid, e = b + per < n ? b + per : n;
    auto cap = [&](int64_t i) -> int64_t {
        const uint64_t len = uint64_t(src_off[i + 1] - src_off[i]);
        if (kDecode) return int64_t((len + 3) / 4 * 3);
        const int a = alph_id ? (alph_id[i] & (kMaxAlphabets - 1)) : 0;
        return int64_t(enc_length(len, tabs.padded[a]));
    };
    int64_t sum = 0;
    for (int64_t i = b; i < e; ++i) sum += cap(i);
    part[tid] = sum;
    __syncthreads();
    for (int o = 1; o < kPrepThreads; o <<= 1) {
        const int64_t v = tid >= o ? part[tid - o] : 0;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    int64_t run = part[tid] - sum;
    for (int64_t i = b; i < e; ++i) {
        dst_off[i] = run;
        run += cap(i);
    }
    if (tid == kPrepThreads - 1) dst_off[n] = part[kPrepThreads - 1];
}

}  // namespace

size_t batch_workspace_bytes(int64_t n) {
    // tile scan (n+1 int64) then one error word per string, 256-byte aligned.
    const size_t scan = (size_t(n) + 1) * sizeof(int64_t);
    return ((scan + 255) & ~size_t(255)) + size_t(n) * sizeof(uint64_t);
}

cudaError_t launch_batch(bool decode, const BatchArgs& a, const BatchTables& tabs, int units,
                         void* workspace, cudaStream_t st) {
    int64_t* tiles = static_cast<int64_t*>(workspace);
    const size_t scan = (size_t(a.n) + 1) * sizeof(int64_t);
    unsigned long long* err = reinterpret_cast<unsigned long long*>(
        static_cast<uint8_t*>(workspace) + ((scan + 255) & ~size_t(255)));
    const uint32_t tile_bytes = uint32_t(32 * units * (decode ? 16 : 12));
    if (decode)
        batch_prep_kernel<true><<<1, kPrepThreads, 0, st>>>(a.src_off, a.n, tile_bytes, tabs,
                                                            a.alph_id, tiles, a.results, err);
    else
        batch_prep_kernel<false><<<1, kPrepThreads, 0, st>>>(a.src_off, a.n, tile_bytes, tabs,
                                                             a.alph_id, tiles, a.results, err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (!decode) {
        switch (units) {
            case 1: return launch_encode_tiles<1>(a, tabs, tiles, st);
            case 2: return launch_encode_tiles<2>(a, tabs, tiles, st);
            case 4: return launch_encode_tiles<4>(a, tabs, tiles, st);
            default: return launch_encode_tiles<8>(a, tabs, tiles, st);
        }
    }
    switch (units) {
        case 1: e = launch_decode_tiles<1>(a, tabs, tiles, err, st); break;
        case 2: e = launch_decode_tiles<2>(a, tabs, tiles, err, st); break;
        case 4: e = launch_decode_tiles<4>(a, tabs, tiles, err, st); break;
        default: e = launch_decode_tiles<8>(a, tabs, tiles, err, st); break;
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
    if (decode)
        batch_offsets_kernel<true><<<1, kPrepThreads, 0, st>>>(src_off, n, tabs, alph_id, dst_off);
    else
        batch_offsets_kernel<false><<<1, kPrepThreads, 0, st>>>(src_off, n, tabs, alph_id, dst_off);
    return cudaGetLastError();
}

}  // namespace b64
