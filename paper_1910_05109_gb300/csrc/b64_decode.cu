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
// that is tested once per chunk by a block-wide vote. Only a chunk that holds
// a bad byte looks for its exact offset (cold path) and folds it into the
// call's result with an atomic minimum.
//
// Fast path (src and dst 16-byte aligned): a persistent grid; each CTA
// streams 16 KiB chunks through a 4-stage ring filled by bulk (TMA) loads,
// writes the 12 KiB of output into a 2-stage shared-memory ring, and stores
// it with bulk (TMA) stores. The body (all but the last 2 to 5 characters) is
// done by this kernel; a one-thread kernel then checks the padding and length
// rules on the tail, decodes it and writes the call's result.
#include <mutex>

#include "b64_internal.h"

namespace b64 {
namespace {

constexpr int kThreads = 256;
constexpr int kUnits = 4;                              // 16-character units per thread
constexpr uint32_t kChunkIn = kThreads * kUnits * 16;  // 16384 characters
constexpr uint32_t kChunkOut = kChunkIn / 4 * 3;       // 12288 bytes
constexpr int kStagesIn = 4;
constexpr int kStagesOut = 2;
constexpr size_t kSmem =
    size_t(kStagesIn) * kChunkIn + size_t(kStagesOut) * kChunkOut + kStagesIn * sizeof(uint64_t);

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

__global__ void __launch_bounds__(kThreads)
    decode_tma_kernel(const uint8_t* __restrict__ src, uint64_t body, uint8_t* __restrict__ dst,
                      const __grid_constant__ DecodeTable tab, unsigned long long* d_err) {
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(16) uint8_t lut[256];
    uint8_t* sin = smem;
    uint8_t* sout = smem + size_t(kStagesIn) * kChunkIn;
    uint64_t* full = reinterpret_cast<uint64_t*>(sout + size_t(kStagesOut) * kChunkOut);

    const int tid = threadIdx.x;
    if (tid < 64) reinterpret_cast<uint32_t*>(lut)[tid] = tab.w[tid];

    const uint64_t n_chunks = body / kChunkIn;
    const uint64_t G = gridDim.x, b = blockIdx.x;
    const uint64_t K = b < n_chunks ? (n_chunks - 1 - b) / G + 1 : 0;

    if (tid == 0) {
        for (int s = 0; s < kStagesIn; ++s) mbar_init(&full[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        for (uint64_t k = 0; k < K && k < kStagesIn; ++k) {
            mbar_arrive_expect_tx(&full[k], kChunkIn);
            bulk_load(sin + k * kChunkIn, src + (b + k * G) * kChunkIn, kChunkIn, &full[k]);
        }
    }

    for (uint64_t k = 0; k < K; ++k) {
        const int s = int(k % kStagesIn);
        const int so = int(k % kStagesOut);
        const uint64_t chunk = b + k * G;
        const bool ok = mbar_wait(&full[s], uint32_t(k / kStagesIn) & 1u);
        // The bulk store that last read sout[so] (kStagesOut chunks ago) must
        // be done reading before the buffer is overwritten.
        if (tid == 0) bulk_wait_read<kStagesOut - 1>();
        __syncthreads();

        const uint4* in = reinterpret_cast<const uint4*>(sin + size_t(s) * kChunkIn);
        uint8_t* out = sout + size_t(so) * kChunkOut;
        uint32_t err = 0;
#pragma unroll
        for (int u = 0; u < kUnits; ++u) {
            const int j = tid + u * kThreads;
            const uint4 c = in[j];
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
        if (__syncthreads_or(int(err & kBad) | int(!ok))) {
            if (__syncthreads_or(!ok)) {
                if (tid == 0) {
                    atomicOr(&g_fault, 1u);
                    for (uint64_t k2 = k + 1; k2 < K && k2 < k + kStagesIn; ++k2)
                        mbar_wait(&full[k2 % kStagesIn], uint32_t(k2 / kStagesIn) & 1u);
                    bulk_wait_read<0>();
                }
                return;
            }
            // Cold path: the exact first bad offset of this chunk.
            uint64_t first = kNoError;
            if (err & kBad) {
                const uint8_t* cin = sin + size_t(s) * kChunkIn;
                for (int u = 0; u < kUnits && first == kNoError; ++u) {
                    const int j = tid + u * kThreads;
                    for (int i = 0; i < 16; ++i) {
                        if (lut[cin[16 * j + i]] & kBad) {
                            first = chunk * kChunkIn + uint64_t(16 * j + i);
                            break;
                        }
                    }
                }
            }
            block_min_to_global(first, d_err);
            // Every warp must be done rescanning sin[s] before thread 0
            // refills it with the next chunk below.
            __syncthreads();
        }
        if (tid == 0) {
            bulk_store(dst + chunk * kChunkOut, out, kChunkOut);
            bulk_commit();
            if (k + kStagesIn < K) {
                mbar_arrive_expect_tx(&full[s], kChunkIn);
                bulk_load(sin + size_t(s) * kChunkIn, src + (b + (k + kStagesIn) * G) * kChunkIn,
                          kChunkIn, &full[s]);
            }
        }
    }
    if (tid == 0) bulk_wait_read<0>();

    if (b == n_chunks % G) {
        const uint64_t first = decode_quads_plain(src, n_chunks * (kChunkIn / 4), body / 4, dst,
                                                  lut, tid, kThreads, true);
        block_min_to_global(first, d_err);
    }
}

__global__ void __launch_bounds__(kThreads)
    decode_generic_kernel(const uint8_t* __restrict__ src, uint64_t body,
                          uint8_t* __restrict__ dst, const __grid_constant__ DecodeTable tab,
                          unsigned long long* d_err) {
    __shared__ __align__(16) uint8_t lut[256];
    if (threadIdx.x < 64) reinterpret_cast<uint32_t*>(lut)[threadIdx.x] = tab.w[threadIdx.x];
    __syncthreads();
    const bool al4 = (reinterpret_cast<uintptr_t>(src) & 3u) == 0;
    const uint64_t first =
        decode_quads_plain(src, 0, body / 4, dst, lut, uint64_t(blockIdx.x) * blockDim.x + threadIdx.x,
                           uint64_t(gridDim.x) * blockDim.x, al4);
    block_min_to_global(first, d_err);
}

__device__ __forceinline__ uint32_t table_at(const DecodeTable& tab, uint32_t c) {
    return (tab.w[c >> 2] >> (8 * (c & 3))) & 0xFFu;
}

// One thread: the padding and length rules on the tail [body, m), the
// tail's bytes, and the call's result (length, or -(first error + 1)).
__global__ void decode_finalize_kernel(const uint8_t* __restrict__ src, uint64_t m,
                                       uint8_t* __restrict__ dst, const __grid_constant__ DecodeTable tab, int padded,
                                       int64_t* d_result) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const uint64_t body = body_length(m);
    uint64_t err = *reinterpret_cast<unsigned long long*>(d_result);
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
    if (err != kNoError) {
        *d_result = -int64_t(err) - 1;
        return;
    }
    // Decode the tail's data characters: groups of four, then a short group
    // of k characters giving k-1 bytes (missing values taken as zero).
    const uint32_t d = tail - pads;
    uint64_t o = body / 4 * 3;
    for (uint32_t j = 0; j < d; j += 4) {
        const uint32_t k = d - j < 4 ? d - j : 4;
        const uint32_t a = v[j], bb = k > 1 ? v[j + 1] : 0u, c = k > 2 ? v[j + 2] : 0u,
                       dd = k > 3 ? v[j + 3] : 0u;
        const uint32_t w = (((a << 6 | bb) << 6 | c) << 6) | dd;
        const uint32_t nb = k == 4 ? 3u : k - 1;
        for (uint32_t t = 0; t < nb; ++t) dst[o++] = uint8_t(w >> (16 - 8 * t));
    }
    *d_result = int64_t(o);
}

struct KernelSetup {
    std::once_flag once;
    cudaError_t err = cudaSuccess;
    int ctas_per_sm = 1;
};
KernelSetup g_setup[64];

}  // namespace

cudaError_t launch_decode(const uint8_t* src, uint64_t m, uint8_t* dst, const DecodeTable& tab,
                          int padded, int64_t* d_result, cudaStream_t stream) {
    const DeviceInfo& di = device_info();
    const uint64_t body = body_length(m);
    unsigned long long* d_err = reinterpret_cast<unsigned long long*>(d_result);
    if (body > 0) {
        const bool aligned =
            ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15u) == 0;
        if (aligned) {
            KernelSetup& ks = g_setup[di.device & 63];
            std::call_once(ks.once, [&] {
                ks.err = cudaFuncSetAttribute(decode_tma_kernel,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              int(kSmem));
                if (ks.err == cudaSuccess)
                    ks.err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                        &ks.ctas_per_sm, decode_tma_kernel, kThreads, kSmem);
                if (ks.ctas_per_sm < 1) ks.ctas_per_sm = 1;
            });
            if (ks.err != cudaSuccess) return ks.err;
            const uint64_t n_chunks = body / kChunkIn;
            uint64_t grid = uint64_t(di.sm_count) * ks.ctas_per_sm;
            if (n_chunks < grid) grid = n_chunks > 0 ? n_chunks : 1;
            decode_tma_kernel<<<unsigned(grid), kThreads, kSmem, stream>>>(src, body, dst, tab,
                                                                             d_err);
        } else {
            const uint64_t quads = body / 4;
            uint64_t grid = (quads + kThreads - 1) / kThreads;
            const uint64_t cap = uint64_t(di.sm_count) * 8;
            if (grid > cap) grid = cap;
            if (grid == 0) grid = 1;
            decode_generic_kernel<<<unsigned(grid), kThreads, 0, stream>>>(src, body, dst, tab,
                                                                             d_err);
        }
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    decode_finalize_kernel<<<1, 32, 0, stream>>>(src, m, dst, tab, padded, d_result);
    return cudaGetLastError();
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
