// Base64 encode kernels (Sec. 2 and Sec. 3.1 of Mula & Lemire).
//
// The paper's AVX-512 loop turns 48 input bytes into 64 characters per
// iteration with one byte gather (vpermb), one multi-shift (vpmultishiftqb)
// and one 64-entry table lookup (vpermb). Here the same three steps run per
// thread on 12-byte units. In the streaming kernel, __byte_perm gathers each
// triple as the 24-bit number s1<<16 | s2<<8 | s3 (Sec. 2), whose two 12-bit
// halves index a 4096-entry table of character pairs built in shared memory
// from the run-time alphabet: two 16-bit lookups and one byte permute give
// the four characters. The plain paths (unaligned buffers, the ragged end)
// build the paper's (s2,s1,s3,s2) word, pick the 6-bit values at bits 10, 4,
// 22 and 16, and look each up in the 64-byte table (16 words in 16 distinct
// banks, so lookups never conflict).
//
// Fast path (src and dst 16-byte aligned): a persistent grid in which every
// warp is its own pipeline. A warp streams "warp chunks" of 32 x kUnits x 12
// input bytes through a ring of kStages shared-memory buffers that its lane 0
// fills with bulk (TMA) copies, each completing on the warp's own mbarrier;
// the lanes turn each chunk into characters. Inputs below 32 MiB use small
// chunks (384 bytes) and many blocks, with coalesced 16-byte stores straight
// to global memory; larger ones use 1152-byte chunks, seven deep, one block
// an SM, and stage the characters in shared memory for bulk stores. No
// block-wide barrier is taken inside the loop, so warps never wait for one
// another. The bytes after the last whole warp chunk and the final 1-2 bytes
// with their padding are done by one warp with plain loads.
#include <mutex>

#include "b64_internal.h"

#ifndef B64_ENC_PAIRS
#define B64_ENC_PAIRS 1
#endif
#ifndef B64_ENC_LARGE_MIN
#define B64_ENC_LARGE_MIN (32ull << 20)
#endif

namespace b64 {
namespace {

// The shape of a streaming encode launch: W warps a block, each with S input
// buffers of 32 x U x 12 bytes filled by bulk copies; with BulkOut the
// characters go through two output buffers a warp and bulk stores, else
// straight to global memory with 16-byte stores.
template <int W, int U, int S, bool BulkOut>
struct EncodeShape {
    static constexpr int kWarps = W;
    static constexpr int kThreads = 32 * W;
    static constexpr int kUnits = U;                      // 12-byte units per lane per chunk
    static constexpr int kStages = S;
    static constexpr int kOutStages = 2;
    static constexpr bool kBulkOut = BulkOut;
    static constexpr uint32_t kChunkIn = 32 * U * 12;     // input bytes per warp chunk
    static constexpr uint32_t kChunkOut = kChunkIn / 3 * 4;
    static constexpr size_t kSmemIn = size_t(W) * S * (kChunkIn + sizeof(uint64_t));
    static constexpr size_t kSmem = kSmemIn + (BulkOut ? size_t(W) * kOutStages * kChunkOut : 0);
    static_assert(kChunkIn % 16 == 0, "bulk copies need 16-byte multiples");
    static_assert(kSmemIn % 16 == 0, "output buffers start on 16-byte boundaries");
    static_assert(kSmem <= 200 * 1024, "shared memory per block, with the pair table");
};
// Below kLargeMin input bytes: 4 blocks an SM of 16 warps with 4 buffers of
// 384 bytes (fine grain for small inputs). From kLargeMin up: one block an SM
// of 16 warps with 7 buffers of 1152 bytes each, 126 KiB of input in flight
// per SM, and bulk stores.
using SmallShape = EncodeShape<16, 1, 4, false>;
using LargeShape = EncodeShape<16, 3, 7, true>;
constexpr uint64_t kLargeMin = B64_ENC_LARGE_MIN;
constexpr int kThreads = 512;                            // generic kernel

__device__ uint32_t g_fault;

__device__ __forceinline__ void store4(uint8_t* p, uint32_t v, bool aligned4) {
    if (aligned4) {
        *reinterpret_cast<uint32_t*>(p) = v;
    } else {
        p[0] = uint8_t(v);
        p[1] = uint8_t(v >> 8);
        p[2] = uint8_t(v >> 16);
        p[3] = uint8_t(v >> 24);
    }
}

// Triples [t_begin, t_end) of src, strided over the calling threads.
__device__ __forceinline__ void encode_triples_plain(const uint8_t* __restrict__ src, uint64_t t_begin,
                                     uint64_t t_end, uint8_t* __restrict__ dst,
                                     const uint8_t* lut, uint64_t tid, uint64_t nthreads,
                                     bool dst_aligned4) {
    for (uint64_t t = t_begin + tid; t < t_end; t += nthreads) {
        const uint8_t* p = src + 3 * t;
        const uint32_t s1 = p[0], s2 = p[1], s3 = p[2];
        const uint32_t g = s2 | (s1 << 8) | (s3 << 16) | (s2 << 24);
        store4(dst + 4 * t, encode_gathered(g, lut), dst_aligned4);
    }
}

// The last n mod 3 bytes: the missing bytes count as zero, and '=' fills the
// group to four characters when padded (Sec. 2).
__device__ __forceinline__ void encode_tail(const uint8_t* __restrict__ src, uint64_t n,
                            uint8_t* __restrict__ dst, const uint8_t* lut, int padded) {
    const uint64_t t = n / 3;
    const uint32_t r = uint32_t(n - 3 * t);
    if (r == 0) return;
    const uint32_t s1 = src[3 * t];
    const uint32_t s2 = r == 2 ? src[3 * t + 1] : 0u;
    const uint32_t g = s2 | (s1 << 8) | (s2 << 24);
    uint8_t* o = dst + 4 * t;
    o[0] = lut[(g >> 10) & 63u];
    o[1] = lut[(g >> 4) & 63u];
    if (r == 2) {
        o[2] = lut[(g >> 22) & 63u];
        if (padded) o[3] = '=';
    } else if (padded) {
        o[2] = '=';
        o[3] = '=';
    }
}


template <class Sh>
__global__ void __launch_bounds__(Sh::kThreads)
    encode_tma_kernel(const uint8_t* __restrict__ src, uint64_t n, uint8_t* __restrict__ dst,
                      const __grid_constant__ EncodeTable tab, int padded) {
    constexpr int kWarps = Sh::kWarps, kThreads = Sh::kThreads, kUnits = Sh::kUnits;
    constexpr int kStages = Sh::kStages, kOutStages = Sh::kOutStages;
    constexpr uint32_t kChunkIn = Sh::kChunkIn, kChunkOut = Sh::kChunkOut;
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(16) uint8_t lut[64];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint8_t* ring = smem + size_t(warp) * kStages * kChunkIn;
    uint64_t* full =
        reinterpret_cast<uint64_t*>(smem + size_t(kWarps) * kStages * kChunkIn) + warp * kStages;

    if (tid < 16) reinterpret_cast<uint32_t*>(lut)[tid] = tab.w[tid];
    if (lane == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
#if B64_ENC_PAIRS
    __shared__ __align__(16) uint16_t pairs[4096];
    build_pairs(pairs, lut, tid, kThreads);
    __syncthreads();
#endif

    const uint64_t n_chunks = n / kChunkIn;
    const uint64_t GW = uint64_t(gridDim.x) * kWarps;
    const uint64_t gw = uint64_t(blockIdx.x) * kWarps + warp;
    const uint64_t K = gw < n_chunks ? (n_chunks - 1 - gw) / GW + 1 : 0;

    if (lane == 0) {
        for (uint64_t k = 0; k < K && k < kStages; ++k) {
            mbar_arrive_expect_tx(&full[k], kChunkIn);
            bulk_load(ring + k * kChunkIn, src + (gw + k * GW) * kChunkIn, kChunkIn, &full[k]);
        }
    }
    for (uint64_t k = 0; k < K; ++k) {
        const int s = int(k % kStages);
        const bool ok = mbar_wait(&full[s], uint32_t(k / kStages) & 1u);
        if (!__all_sync(0xffffffffu, ok)) {
            // A bulk copy did not arrive in time: flag it, let the copies in
            // flight land (bounded), and stop this warp.
            if (lane == 0) {
                atomicOr(&g_fault, 1u);
                for (uint64_t k2 = k; k2 < K && k2 < k + kStages; ++k2)
                    mbar_wait(&full[k2 % kStages], uint32_t(k2 / kStages) & 1u);
                if constexpr (Sh::kBulkOut) bulk_wait_read<0>();
            }
            return;
        }
        const uint8_t* in = ring + size_t(s) * kChunkIn;
        uint8_t* const sbuf =
            Sh::kBulkOut ? smem + Sh::kSmemIn + (size_t(warp) * kOutStages + k % kOutStages) * kChunkOut
                         : nullptr;
        uint4* out = reinterpret_cast<uint4*>(dst + (gw + k * GW) * kChunkOut);
        if constexpr (Sh::kBulkOut) {
            // the bulk store that last read this buffer is done reading it
            if (lane == 0) bulk_wait_read<kOutStages - 1>();
            __syncwarp();
            out = reinterpret_cast<uint4*>(sbuf);
        }
#pragma unroll
        for (int u = 0; u < kUnits; ++u) {
            const int j = lane + 32 * u;
            const uint32_t* w = reinterpret_cast<const uint32_t*>(in + 12 * j);
#if B64_ENC_PAIRS
            out[j] = encode12_pairs(w[0], w[1], w[2], pairs);
#else
            out[j] = encode12(w[0], w[1], w[2], lut);
#endif
        }
        if constexpr (Sh::kBulkOut) {
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                bulk_store(dst + (gw + k * GW) * kChunkOut, sbuf, kChunkOut);
                bulk_commit();
            }
        }
        __syncwarp();
        if (lane == 0 && k + kStages < K) {
            mbar_arrive_expect_tx(&full[s], kChunkIn);
            bulk_load(ring + size_t(s) * kChunkIn, src + (gw + (k + kStages) * GW) * kChunkIn,
                      kChunkIn, &full[s]);
        }
    }

    if constexpr (Sh::kBulkOut) {
        if (lane == 0) bulk_wait_read<0>();
    }
    if (gw == n_chunks % GW) {
        encode_triples_plain(src, n_chunks * (kChunkIn / 3), n / 3, dst, lut, lane, 32, true);
        if (lane == 0) encode_tail(src, n, dst, lut, padded);
    }
}

__global__ void __launch_bounds__(kThreads)
    encode_generic_kernel(const uint8_t* __restrict__ src, uint64_t n, uint8_t* __restrict__ dst,
                          const __grid_constant__ EncodeTable tab, int padded) {
    __shared__ __align__(16) uint8_t lut[64];
    if (threadIdx.x < 16) reinterpret_cast<uint32_t*>(lut)[threadIdx.x] = tab.w[threadIdx.x];
    __syncthreads();
    // the tail first: nothing of it then stays live across the loop below
    if (blockIdx.x == 0 && threadIdx.x == 0) encode_tail(src, n, dst, lut, padded);
    const bool al4 = (reinterpret_cast<uintptr_t>(dst) & 3u) == 0;
    encode_triples_plain(src, 0, n / 3, dst, lut, uint64_t(blockIdx.x) * blockDim.x + threadIdx.x,
                         uint64_t(gridDim.x) * blockDim.x, al4);
}

struct KernelSetup {
    std::once_flag once;
    cudaError_t err = cudaSuccess;
    int ctas_per_sm = 1;
};
KernelSetup g_small[64], g_large[64];

// One resident grid of encode_tma_kernel<Sh> (fewer blocks when the input
// has fewer chunks than the grid has warps).
template <class Sh>
cudaError_t launch_tma(KernelSetup& ks, const uint8_t* src, uint64_t n, uint8_t* dst,
                       const EncodeTable& tab, int padded, cudaStream_t stream) {
    const DeviceInfo& di = device_info();
    std::call_once(ks.once, [&] {
        ks.err = cudaFuncSetAttribute(encode_tma_kernel<Sh>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, int(Sh::kSmem));
        if (ks.err == cudaSuccess)
            ks.err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &ks.ctas_per_sm, encode_tma_kernel<Sh>, Sh::kThreads, Sh::kSmem);
        if (ks.ctas_per_sm < 1) ks.ctas_per_sm = 1;
    });
    if (ks.err != cudaSuccess) return ks.err;
    const uint64_t n_chunks = n / Sh::kChunkIn;
    const uint64_t want = (n_chunks + Sh::kWarps - 1) / Sh::kWarps;
    uint64_t grid = uint64_t(di.sm_count) * ks.ctas_per_sm;
    if (want < grid) grid = want > 0 ? want : 1;
    encode_tma_kernel<Sh><<<unsigned(grid), Sh::kThreads, Sh::kSmem, stream>>>(src, n, dst, tab,
                                                                              padded);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_encode(const uint8_t* src, uint64_t n, uint8_t* dst, const EncodeTable& tab,
                          int padded, cudaStream_t stream) {
    const DeviceInfo& di = device_info();
    const bool aligned = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) &
                          15u) == 0;
    if (aligned) {
        return n >= kLargeMin
                   ? launch_tma<LargeShape>(g_large[di.device & 63], src, n, dst, tab, padded, stream)
                   : launch_tma<SmallShape>(g_small[di.device & 63], src, n, dst, tab, padded, stream);
    }
    const uint64_t triples = n / 3;
    uint64_t grid = (triples + kThreads - 1) / kThreads;
    const uint64_t cap = uint64_t(di.sm_count) * 8;
    if (grid > cap) grid = cap;
    if (grid == 0) grid = 1;
    encode_generic_kernel<<<unsigned(grid), kThreads, 0, stream>>>(src, n, dst, tab, padded);
    return cudaGetLastError();
}

uint32_t encode_fault_flag(bool clear) {
    uint32_t v = 0;
    cudaMemcpyFromSymbol(&v, g_fault, sizeof(v));
    if (clear && v) {
        const uint32_t z = 0;
        cudaMemcpyToSymbol(g_fault, &z, sizeof(z));
    }
    return v;
}

}  // namespace b64
