// Strict base64 decode kernels (Sec. 2 and Sec. 3.2 of Mula & Lemire).
//
// The paper's AVX-512 loop turns 64 characters into 48 bytes per iteration:
// a 128-entry table lookup maps characters to 6-bit values (0x80 for
// anything outside the alphabet), the input and the looked-up values are ORed
// into an error register that is tested once per stream (Fig. 2), two
// multiply-adds merge four 6-bit values into 24 bits, and a byte permutation
// packs the 24-bit words. Here each thread does the same on 16-character
// units: byte lookups in a 256-entry shared-memory table (entries >= 0x80 are
// all 0x80, which folds in the test of the input's top bit), shifts and ORs
// for the merge, __byte_perm for the pack, and an OR-accumulated error word
// that is tested once per chunk by a warp-wide vote. Only a chunk that holds
// a bad byte looks for its exact offset (cold path) and folds it into the
// call's result with an atomic minimum.
//
// Body path (src and dst 16-byte aligned): a persistent grid of one 16-warp
// block an SM in which every warp works alone on "warp chunks" of
// 32 x kUnits x 16 characters. Lane 0 of each warp keeps kStagesIn bulk (TMA)
// copies of its next chunks in flight into a per-warp ring of shared-memory
// buffers; the warp decodes a landed chunk from shared memory (16 characters
// a lane), writes the 12-byte results into one of kStagesOut output buffers,
// and lane 0 stores that buffer with a bulk store and refills the input
// buffer. Inputs of 64 MiB and more use 1 KiB chunks eight deep (128 KiB of
// input in flight per SM, at 32 registers a thread); smaller ones use 2 KiB
// chunks four deep. The error vote and the cold-path search are warp-wide,
// so no block-wide barrier is taken inside the loop. The body (all but the
// last 2 to 5 characters) is done by this kernel; a one-thread kernel then
// checks the padding and length rules on the tail, decodes it and writes the
// call's result.
#include <mutex>

#include <cooperative_groups.h>

#include "b64_internal.h"

#ifndef B64_DEC_LARGE_MIN
#define B64_DEC_LARGE_MIN (64ull << 20)
#endif

namespace b64 {
namespace {

// The shape of a body launch: W warps a block, each with SI input buffers of
// 32 x U x 16 characters filled by bulk copies and SO output buffers.
template <int W, int U, int SI, int SO>
struct DecodeShape {
    static constexpr int kWarps = W;
    static constexpr int kThreads = 32 * W;
    static constexpr int kUnits = U;                     // 16-character units per lane per chunk
    static constexpr int kStagesIn = SI;
    static constexpr int kStagesOut = SO;
    static constexpr uint32_t kChunkIn = 32 * U * 16;    // characters per warp chunk
    static constexpr uint32_t kChunkOut = kChunkIn / 4 * 3;
    // per warp: SI input and SO output buffers; then one barrier per input buffer
    static constexpr size_t kSmemRings = size_t(W) * (size_t(SI) * kChunkIn + size_t(SO) * kChunkOut);
    static constexpr size_t kSmem = kSmemRings + size_t(W) * SI * sizeof(uint64_t);
    static_assert(kChunkOut % 16 == 0, "bulk copies need 16-byte multiples");
    static_assert(kSmem <= 227 * 1024, "shared memory per block");
};
// One 16-warp block an SM. Below kLargeMin characters: 2 KiB chunks, four
// deep (fewer bulk copies per byte, which pays when the input is in L2).
// From kLargeMin up: 1 KiB chunks, eight deep, 128 KiB in flight per SM (the
// faster shape for inputs streamed from DRAM).
using SmallShape = DecodeShape<16, 4, 4, 2>;
using LargeShape = DecodeShape<16, 2, 8, 2>;
constexpr uint64_t kLargeMin = B64_DEC_LARGE_MIN;
constexpr int kThreads = 512;                            // generic kernel
// A body kernel whose bulk copy did not arrive folds this into the result
// word instead of an offset (offsets are below 2^62); the tail kernel turns
// it into B64_E_TIMEOUT.
constexpr uint64_t kTimedOut = uint64_t(1) << 62;
__device__ uint32_t g_fault;

// Characters [0, body) are whole groups of four that cannot contain valid
// padding; the last 2..5 characters (all of them when m < 6) are the tail.
__host__ __device__ __forceinline__ uint64_t body_length(uint64_t m) {
    return m >= 2 ? ((m - 2) & ~uint64_t(3)) : 0;
}

__device__ __forceinline__ uint32_t load4(const uint8_t* p, bool aligned4) {
    if (aligned4) return *reinterpret_cast<const uint32_t*>(p);
    return uint32_t(p[0]) | (uint32_t(p[1]) << 8) | (uint32_t(p[2]) << 16) |
           (uint32_t(p[3]) << 24);
}

// Quads [q_begin, q_end), strided over the calling threads. Returns this
// thread's smallest bad offset (kNoError if none).
__device__ __forceinline__ uint64_t decode_quads_plain(const uint8_t* __restrict__ src, uint64_t q_begin,
                                       uint64_t q_end, uint8_t* __restrict__ dst,
                                       const uint8_t* lut, uint64_t tid, uint64_t nthreads,
                                       bool src_aligned4) {
    uint64_t first = kNoError;
    for (uint64_t q = q_begin + tid; q < q_end; q += nthreads) {
        const uint32_t w = load4(src + 4 * q, src_aligned4);
        uint32_t err = 0;
        const uint32_t v = decode4(w, lut, err);
        if (err & kBad) {
            for (int i = 0; i < 4; ++i) {
                if (lut[(w >> (8 * i)) & 0xFFu] & kBad) {
                    const uint64_t pos = 4 * q + i;
                    first = pos < first ? pos : first;
                    break;
                }
            }
        } else {
            uint8_t* o = dst + 3 * q;
            o[0] = uint8_t(v >> 16);
            o[1] = uint8_t(v >> 8);
            o[2] = uint8_t(v);
        }
    }
    return first;
}

// Folds per-thread first-error offsets into *d_err (all threads of the block
// must call it).
__device__ void block_min_to_global(uint64_t first, unsigned long long* d_err) {
    const uint64_t w = warp_min_u64(first);
    if ((threadIdx.x & 31) == 0 && w != kNoError) atomicMin(d_err, (unsigned long long)w);
}

// One thread: *d_err = "no error" before the body kernel folds offsets into it.
__global__ void result_init_kernel(unsigned long long* d_err) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *d_err = kNoError;
}

__device__ __forceinline__ int first_bad_in(uint32_t w, const uint8_t* lut) {
    for (int i = 0; i < 4; ++i)
        if (lut[(w >> (8 * i)) & 0xFFu] & kBad) return i;
    return -1;
}

template <class Sh>
__global__ void __launch_bounds__(Sh::kThreads)
    decode_body_kernel(const uint8_t* __restrict__ src, uint64_t body, uint8_t* __restrict__ dst,
                       const __grid_constant__ DecodeTable tab, unsigned long long* d_err) {
    constexpr int kWarps = Sh::kWarps, kUnits = Sh::kUnits;
    constexpr int kStagesIn = Sh::kStagesIn, kStagesOut = Sh::kStagesOut;
    constexpr uint32_t kChunkIn = Sh::kChunkIn, kChunkOut = Sh::kChunkOut;
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(16) uint8_t lut[256];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint8_t* ring = smem + size_t(warp) * kStagesIn * kChunkIn;
    uint8_t* sout =
        smem + size_t(kWarps) * kStagesIn * kChunkIn + size_t(warp) * kStagesOut * kChunkOut;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + Sh::kSmemRings) + warp * kStagesIn;
    if (tid < 64) reinterpret_cast<uint32_t*>(lut)[tid] = tab.w[tid];
    if (lane == 0) {
        for (int s = 0; s < kStagesIn; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    wait_prior_grid();  // *d_err has been initialised

    const uint64_t n_chunks = body / kChunkIn;
    const uint64_t GW = uint64_t(gridDim.x) * kWarps;
    const uint64_t gw = uint64_t(blockIdx.x) * kWarps + warp;
    const uint64_t K = gw < n_chunks ? (n_chunks - 1 - gw) / GW + 1 : 0;
    auto chunk_at = [&](uint64_t k) { return gw + k * GW; };

    if (lane == 0) {
        for (uint64_t k = 0; k < K && k < uint64_t(kStagesIn); ++k) {
            mbar_arrive_expect_tx(&full[k], kChunkIn);
            bulk_load(ring + k * kChunkIn, src + chunk_at(k) * kChunkIn, kChunkIn, &full[k]);
        }
    }
    for (uint64_t k = 0; k < K; ++k) {
        const uint64_t chunk = chunk_at(k);
        const int s = int(k % kStagesIn);
        const bool ok = mbar_wait(&full[s], uint32_t(k / kStagesIn) & 1u);
        if (!__all_sync(0xffffffffu, ok)) {
            // A bulk copy did not arrive in time: flag it, let the copies in
            // flight land (bounded), and stop this warp.
            if (lane == 0) {
                atomicOr(&g_fault, 1u);
                atomicMin(d_err, (unsigned long long)kTimedOut);
                for (uint64_t k2 = k; k2 < K && k2 < k + kStagesIn; ++k2)
                    mbar_wait(&full[k2 % kStagesIn], uint32_t(k2 / kStagesIn) & 1u);
                bulk_wait_read<0>();
            }
            return;
        }
        const uint8_t* in = ring + size_t(s) * kChunkIn;
        // The bulk store that last read this output buffer (kStagesOut chunks
        // ago) must be done reading it before it is overwritten.
        const int so = int(k % kStagesOut);
        if (lane == 0) bulk_wait_read<kStagesOut - 1>();
        __syncwarp();
        uint8_t* out = sout + size_t(so) * kChunkOut;
        uint32_t err = 0;
#pragma unroll
        for (int u = 0; u < kUnits; ++u) {
            const int j = lane + 32 * u;
            const uint4 c = *reinterpret_cast<const uint4*>(in + 16 * j);
            const uint32_t q0 = decode4(c.x, lut, err);
            const uint32_t q1 = decode4(c.y, lut, err);
            const uint32_t q2 = decode4(c.z, lut, err);
            const uint32_t q3 = decode4(c.w, lut, err);
            const uint3 o = pack4x24(q0, q1, q2, q3);
            uint32_t* ow = reinterpret_cast<uint32_t*>(out + 12 * j);
            ow[0] = o.x;
            ow[1] = o.y;
            ow[2] = o.z;
        }
        fence_proxy_async_smem();
        if (__any_sync(0xffffffffu, err & kBad)) {
            // Cold path: the exact first bad offset of this warp chunk, from
            // the characters still in the input buffer.
            uint64_t first = kNoError;
            for (int u = 0; u < kUnits && first == kNoError; ++u) {
                const uint32_t* w4 = reinterpret_cast<const uint32_t*>(in + 16 * (lane + 32 * u));
                for (int q = 0; q < 4 && first == kNoError; ++q) {
                    const int i = first_bad_in(w4[q], lut);
                    if (i >= 0)
                        first = chunk * kChunkIn + uint64_t(16 * (lane + 32 * u) + 4 * q + i);
                }
            }
            const uint64_t w = warp_min_u64(first);
            if (lane == 0 && w != kNoError) atomicMin(d_err, (unsigned long long)w);
        }
        __syncwarp();  // every lane is done with `in` and has written `out`
        if (lane == 0) {
            bulk_store(dst + chunk * kChunkOut, out, kChunkOut);
            bulk_commit();
            if (k + kStagesIn < K) {
                mbar_arrive_expect_tx(&full[s], kChunkIn);
                bulk_load(ring + size_t(s) * kChunkIn, src + chunk_at(k + kStagesIn) * kChunkIn,
                          kChunkIn, &full[s]);
            }
        }
    }
    if (lane == 0) bulk_wait_read<0>();

    if (gw == n_chunks % GW) {
        const uint64_t first = decode_quads_plain(src, n_chunks * (kChunkIn / 4), body / 4, dst,
                                                  lut, lane, 32, true);
        const uint64_t w = warp_min_u64(first);
        if (lane == 0 && w != kNoError) atomicMin(d_err, (unsigned long long)w);
    }
}

__global__ void __launch_bounds__(kThreads)
    decode_generic_kernel(const uint8_t* __restrict__ src, uint64_t body,
                          uint8_t* __restrict__ dst, const __grid_constant__ DecodeTable tab,
                          unsigned long long* d_err) {
    __shared__ __align__(16) uint8_t lut[256];
    if (threadIdx.x < 64) reinterpret_cast<uint32_t*>(lut)[threadIdx.x] = tab.w[threadIdx.x];
    __syncthreads();
    wait_prior_grid();  // *d_err has been initialised
    const bool al4 = (reinterpret_cast<uintptr_t>(src) & 3u) == 0;
    const uint64_t first =
        decode_quads_plain(src, 0, body / 4, dst, lut, uint64_t(blockIdx.x) * blockDim.x + threadIdx.x,
                           uint64_t(gridDim.x) * blockDim.x, al4);
    block_min_to_global(first, d_err);
}

__device__ __forceinline__ uint32_t table_at(const DecodeTable& tab, uint32_t c) {
    return (tab.w[c >> 2] >> (8 * (c & 3))) & 0xFFu;
}

// The padding and length rules on the tail [body, m) (one thread), given the
// smallest bad offset found in the body (kNoError if none): writes the
// tail's bytes and returns the call's result (length, or -(first error + 1)).
__device__ int64_t tail_result(const uint8_t* __restrict__ src, uint64_t m,
                               uint8_t* __restrict__ dst, const DecodeTable& tab, int flags,
                               uint64_t err) {
    const bool padded = flags & 1, canonical = flags & 2;
    const uint64_t body = body_length(m);
    const uint32_t last = m >= 1 ? src[m - 1] : 0u;
    uint32_t pads = 0;
    if (padded && m >= 1 && last == '=') pads = (m >= 2 && src[m - 2] == '=') ? 2 : 1;

    uint32_t v[5] = {0, 0, 0, 0, 0};
    const uint32_t tail = uint32_t(m - body);
    for (uint32_t i = 0; i < tail; ++i) {
        const uint64_t pos = body + i;
        const uint32_t ch = src[pos];
        v[i] = table_at(tab, ch);
        if (v[i] & kBad) {
            const bool pad_ok =
                padded && ch == '=' && (pos == m - 1 || (pos + 2 == m && last == '='));
            if (!pad_ok) {
                err = pos < err ? pos : err;
                break;
            }
        }
    }
    if (padded ? (m % 4 != 0) : (m % 4 == 1)) err = m < err ? m : err;
    const uint32_t d = tail - pads;
    if (canonical && (d % 4 == 2 || d % 4 == 3)) {
        // the last data character's bits that reach no output byte must be zero
        const uint32_t last_v = v[d - 1], low = d % 4 == 2 ? 15u : 3u;
        const uint64_t pos = body + d - 1;
        if (!(last_v & kBad) && (last_v & low)) err = pos < err ? pos : err;
    }
    if (err != kNoError) return -int64_t(err) - 1;
    // Decode the tail's data characters: groups of four, then a short group
    // of k characters giving k-1 bytes (missing values taken as zero).
    uint64_t o = body / 4 * 3;
    for (uint32_t j = 0; j < d; j += 4) {
        const uint32_t k = d - j < 4 ? d - j : 4;
        const uint32_t a = v[j], bb = k > 1 ? v[j + 1] : 0u, c = k > 2 ? v[j + 2] : 0u,
                       dd = k > 3 ? v[j + 3] : 0u;
        const uint32_t w = (((a << 6 | bb) << 6 | c) << 6) | dd;
        const uint32_t nb = k == 4 ? 3u : k - 1;
        for (uint32_t t = 0; t < nb; ++t) dst[o++] = uint8_t(w >> (16 - 8 * t));
    }
    return int64_t(o);
}

// One thread: the tail rules after the body kernels have folded their first
// bad offset into *d_result.
__global__ void decode_finalize_kernel(const uint8_t* __restrict__ src, uint64_t m,
                                       uint8_t* __restrict__ dst, const __grid_constant__ DecodeTable tab, int flags,
                                       int64_t* d_result) {
    wait_prior_grid();  // the body kernel has folded in its offsets
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const uint64_t err = *reinterpret_cast<unsigned long long*>(d_result);
    *d_result = err == kTimedOut ? B64_E_TIMEOUT : tail_result(src, m, dst, tab, flags, err);
}

// Inputs of at most kSmallMax characters: the whole strict decode in one
// launch of one cluster of up to kSmallCtas blocks (no result
// initialisation, no separate tail kernel). Every thread loads all of its
// groups before decoding any of them; each block folds its first bad offset
// into its shared memory, and after a cluster barrier block 0 reads the
// others' through distributed shared memory and applies the tail rules.
// One block up to kSmallSingle characters; above, a cluster of one block per
// kSmallCtaBytes, at most kSmallCtas blocks (16, a non-portable cluster size,
// where the device can co-schedule it; else 8). Measured in CUDA graphs: a
// 188 KB input in 5.2 us with 16 blocks against 7.1 us with three 64 KiB
// blocks.
constexpr int kSmallThreads = 1024;
constexpr int kSmallPer = 16;                                   // groups per thread, at most
constexpr int kSmallCtas = 16;
constexpr uint64_t kSmallPerCta = uint64_t(kSmallThreads) * kSmallPer * 4;  // 64 KiB
constexpr uint64_t kSmallMax = kSmallPerCta * 8;                            // 512 KiB
constexpr uint64_t kSmallSingle = 32u << 10;
constexpr uint64_t kSmallCtaBytes = 8u << 10;

template <bool kCluster>
__global__ void __launch_bounds__(kSmallThreads)
    decode_small_kernel(const uint8_t* __restrict__ src, uint64_t m, uint8_t* __restrict__ dst,
                        const __grid_constant__ DecodeTable tab, int flags, int64_t* d_result) {
    namespace cg = cooperative_groups;
    __shared__ __align__(16) uint8_t lut[256];
    __shared__ unsigned long long s_err;
    const int tid = threadIdx.x;
    const uint32_t rank = kCluster ? cg::this_cluster().block_rank() : 0u;
    const uint32_t nblocks = kCluster ? cg::this_cluster().num_blocks() : 1u;
    if (tid < 64) reinterpret_cast<uint32_t*>(lut)[tid] = tab.w[tid];
    if (tid == 0) s_err = kNoError;
    __syncthreads();
    const uint64_t quads = body_length(m) / 4;
    const bool al4 = (reinterpret_cast<uintptr_t>(src) & 3u) == 0;
    const uint64_t g = uint64_t(rank) * kSmallThreads + tid, stride = uint64_t(nblocks) * kSmallThreads;
    uint32_t w[kSmallPer];
#pragma unroll
    for (int k = 0; k < kSmallPer; ++k) {
        const uint64_t q = g + uint64_t(k) * stride;
        w[k] = q < quads ? load4(src + 4 * q, al4) : 0x41414141u;  // "AAAA": valid filler
    }
    uint64_t first = kNoError;
#pragma unroll
    for (int k = 0; k < kSmallPer; ++k) {
        const uint64_t q = g + uint64_t(k) * stride;
        if (q >= quads) break;
        uint32_t err = 0;
        const uint32_t v = decode4(w[k], lut, err);
        if (err & kBad) {
            for (int i = 0; i < 4; ++i) {
                if (lut[(w[k] >> (8 * i)) & 0xFFu] & kBad) {
                    const uint64_t pos = 4 * q + i;
                    first = pos < first ? pos : first;
                    break;
                }
            }
        } else {
            uint8_t* o = dst + 3 * q;
            o[0] = uint8_t(v >> 16);
            o[1] = uint8_t(v >> 8);
            o[2] = uint8_t(v);
        }
    }
    const uint64_t wmin = warp_min_u64(first);
    if ((tid & 31) == 0 && wmin != kNoError) atomicMin(&s_err, (unsigned long long)wmin);
    if (!kCluster) {
        __syncthreads();
        if (tid == 0) *d_result = tail_result(src, m, dst, tab, flags, s_err);
        return;
    }
    cg::cluster_group cluster = cg::this_cluster();
    cluster.sync();  // every block's minimum (and bytes) are final
    if (rank == 0 && tid == 0) {
        uint64_t err = kNoError;
        for (uint32_t r = 0; r < nblocks; ++r) {
            const uint64_t e = *cluster.map_shared_rank(&s_err, r);
            err = e < err ? e : err;
        }
        *d_result = tail_result(src, m, dst, tab, flags, err);
    }
    cluster.sync();  // no block leaves while block 0 may still read its shared memory
}

struct KernelSetup {
    std::once_flag once;
    cudaError_t err = cudaSuccess;
    int ctas_per_sm = 1;
};
KernelSetup g_small[64], g_large[64];

// Launches a persistent body kernel (warps x chunk characters per warp
// chunk) as a programmatic dependent: one grid of resident CTAs, fewer when
// the body has fewer chunks than warps.
template <class Kernel>
cudaError_t launch_body(Kernel kernel, KernelSetup& ks, int threads, size_t smem, uint32_t chunk,
                        const uint8_t* src, uint64_t body, uint8_t* dst, const DecodeTable& tab,
                        unsigned long long* d_err, cudaStream_t stream) {
    const DeviceInfo& di = device_info();
    std::call_once(ks.once, [&] {
        ks.err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (ks.err == cudaSuccess)
            ks.err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ks.ctas_per_sm, kernel, threads, smem);
        if (ks.ctas_per_sm < 1) ks.ctas_per_sm = 1;
    });
    if (ks.err != cudaSuccess) return ks.err;
    const uint64_t warps = uint64_t(threads / 32);
    const uint64_t want = (body / chunk + warps - 1) / warps;
    uint64_t grid = uint64_t(di.sm_count) * ks.ctas_per_sm;
    if (want < grid) grid = want > 0 ? want : 1;
    return launch_dependent(kernel, unsigned(grid), threads, smem, stream, src, body, dst, tab, d_err);
}

struct ClusterLimit {
    std::once_flag once;
    int ctas = 8;
};
ClusterLimit g_small_limit[64];

// The largest cluster of the small-input kernel this device co-schedules:
// kSmallCtas if it allows that non-portable size, else the portable 8.
int small_cluster_limit() {
    int dev = 0;
    cudaGetDevice(&dev);
    ClusterLimit& cl = g_small_limit[dev & 63];
    std::call_once(cl.once, [&] {
        if (cudaFuncSetAttribute(decode_small_kernel<true>,
                                 cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        cudaLaunchConfig_t c = {};
        c.gridDim = dim3(kSmallCtas);
        c.blockDim = dim3(kSmallThreads);
        int size = 0;
        if (cudaOccupancyMaxPotentialClusterSize(&size, decode_small_kernel<true>, &c) !=
            cudaSuccess) {
            cudaGetLastError();
            return;
        }
        if (size > 8) cl.ctas = size < kSmallCtas ? size : kSmallCtas;
    });
    return cl.ctas;
}

}  // namespace

cudaError_t launch_decode(const uint8_t* src, uint64_t m, uint8_t* dst, const DecodeTable& tab,
                          int flags, int64_t* d_result, cudaStream_t stream) {
    if (m <= kSmallMax) {
        const int max_ctas = small_cluster_limit();
        uint64_t want = (m + kSmallCtaBytes - 1) / kSmallCtaBytes;
        if (want > uint64_t(max_ctas)) want = uint64_t(max_ctas);
        // m <= 8 blocks x kSmallPerCta, so 8 blocks always hold every group
        const unsigned ctas = unsigned(m <= kSmallSingle ? 1 : (want < 2 ? 2 : want));
        if (ctas == 1) {
            decode_small_kernel<false><<<1, kSmallThreads, 0, stream>>>(src, m, dst, tab, flags,
                                                                        d_result);
            return cudaGetLastError();
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(ctas);
        cfg.blockDim = dim3(kSmallThreads);
        cfg.stream = stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = ctas;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, decode_small_kernel<true>, src, m, dst, tab, flags,
                                  d_result);
    }
    const DeviceInfo& di = device_info();
    const uint64_t body = body_length(m);
    unsigned long long* d_err = reinterpret_cast<unsigned long long*>(d_result);
    // the body kernels fold their first bad offsets into *d_result: start at
    // "none"; the body and tail kernels are programmatic dependents, so their
    // launches overlap the kernel before them
    result_init_kernel<<<1, 32, 0, stream>>>(d_err);
    const cudaError_t e0 = cudaGetLastError();
    if (e0 != cudaSuccess) return e0;
    if (body > 0) {
        const bool aligned =
            ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15u) == 0;
        if (aligned) {
            const int dv = di.device & 63;
            const cudaError_t e1 =
                body >= kLargeMin
                    ? launch_body(decode_body_kernel<LargeShape>, g_large[dv], LargeShape::kThreads,
                                  LargeShape::kSmem, LargeShape::kChunkIn, src, body, dst, tab, d_err,
                                  stream)
                    : launch_body(decode_body_kernel<SmallShape>, g_small[dv], SmallShape::kThreads,
                                  SmallShape::kSmem, SmallShape::kChunkIn, src, body, dst, tab, d_err,
                                  stream);
            if (e1 != cudaSuccess) return e1;
        } else {
            const uint64_t quads = body / 4;
            uint64_t grid = (quads + kThreads - 1) / kThreads;
            const uint64_t cap = uint64_t(di.sm_count) * 8;
            if (grid > cap) grid = cap;
            if (grid == 0) grid = 1;
            const cudaError_t e1 = launch_dependent(decode_generic_kernel, unsigned(grid), kThreads,
                                                    0, stream, src, body, dst, tab, d_err);
            if (e1 != cudaSuccess) return e1;
        }
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return launch_dependent(decode_finalize_kernel, 1, 32, 0, stream, src, m, dst, tab, flags,
                            d_result);
}


uint32_t decode_fault_flag(bool clear) {
    uint32_t v = 0;
    cudaMemcpyFromSymbol(&v, g_fault, sizeof(v));
    if (clear && v) {
        const uint32_t z = 0;
        cudaMemcpyToSymbol(g_fault, &z, sizeof(z));
    }
    return v;
}

}  // namespace b64
