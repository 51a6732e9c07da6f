// Device-side building blocks shared by the codec kernels: lookup-table
// parameter blocks, the byte-level encode/decode steps, and thin inline-PTX
// wrappers for mbarriers and bulk (TMA) copies on sm_103a.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#ifndef B64_JOIN_WITH_PRMT
#define B64_JOIN_WITH_PRMT 1
#endif

namespace b64 {

// ------------------------------------------------------------------ tables
// The alphabet travels by value in the kernel parameters, so a launch needs
// no device allocation and can be recorded in a CUDA graph.

// 64 output characters indexed by a 6-bit value (Table 1 or any other
// run-time table, Sec. 3.1).
struct EncodeTable {
    uint32_t w[16];
};

// 256 entries indexed by an input byte: the 6-bit value of an alphabet
// character, 0x80 for every other byte (Sec. 3.2 uses 128 entries and ORs the
// input's top bit into the error; indexing by the whole byte folds that OR
// into the table: entries 128..255 are all 0x80).
struct DecodeTable {
    uint32_t w[64];
};

constexpr uint32_t kBad = 0x80u;
constexpr uint64_t kNoError = ~0ull;

// Bounded waits give up after this many nanoseconds of %globaltimer.
constexpr uint64_t kWaitLimitNs = 2000000000ull;

// Joins four bytes (each < 256) into a word, c0 in the low byte: three byte
// permutes, or (B64_JOIN_WITH_PRMT=0) three multiply-adds on the FMA pipe.
__device__ __forceinline__ uint32_t join4(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3) {
#if B64_JOIN_WITH_PRMT
    return __byte_perm(__byte_perm(c0, c1, 0x7740u), __byte_perm(c2, c3, 0x7740u), 0x5410u);
#else
    return (c3 * 256u + c2) * 65536u + (c1 * 256u + c0);
#endif
}

// ------------------------------------------------------------------ encode step
// Sec. 3.1: a triple (s1,s2,s3) is first spread into the 32-bit word whose
// bytes, lowest first, are (s2,s1,s3,s2); then the four 6-bit values sit at
// bit offsets 10, 4, 22 and 16 of that word. `g` is that word.
__device__ __forceinline__ uint32_t encode_gathered(uint32_t g, const uint8_t* lut) {
    const uint32_t c0 = lut[(g >> 10) & 63u];
    const uint32_t c1 = lut[(g >> 4) & 63u];
    const uint32_t c2 = lut[(g >> 22) & 63u];
    const uint32_t c3 = lut[(g >> 16) & 63u];
    return join4(c0, c1, c2, c3);
}

#ifndef B64_ENC_VARIANT
#define B64_ENC_VARIANT 1
#endif

// Sec. 2 as a 24-bit number: v = s1<<16 | s2<<8 | s3, whose four 6-bit
// fields from the top are the four values. The outer fields need one
// instruction each when the top byte is clean (v >> 18, v & 63); the middle
// two are taken either with shift-and-mask
// (ALU pipe) or with a multiply and a multiply-high (FMA pipe), to balance
// the two pipes.
// kClean: the top byte of v is zero (otherwise the first field is masked).
template <bool kClean>
__device__ __forceinline__ uint32_t encode_v24(uint32_t v, const uint8_t* lut) {
    const uint32_t c0 = lut[kClean ? v >> 18 : (v >> 18) & 63u];
#if B64_ENC_VARIANT == 2
    const uint32_t c1 = lut[__umulhi(v * 16384u, 64u)];
    const uint32_t c2 = lut[__umulhi(v * 1048576u, 64u)];
#else
    const uint32_t c1 = lut[(v >> 12) & 63u];
    const uint32_t c2 = lut[(v >> 6) & 63u];
#endif
    const uint32_t c3 = lut[v & 63u];
    return join4(c0, c1, c2, c3);
}

// Encodes 12 bytes held in three little-endian words (x = bytes 0..3,
// y = 4..7, z = 8..11) into 16 characters, returned as four words. Variant 0:
// the __byte_perm selectors pick (s2,s1,s3,s2) of each of the four triples
// (the paper's gather, Sec. 3.1); variants 1, 2: they pick (s3,s2,s1,0), the
// triple as a big-endian 24-bit number.
__device__ __forceinline__ uint4 encode12(uint32_t x, uint32_t y, uint32_t z, const uint8_t* lut) {
    uint4 o;
#if B64_ENC_VARIANT == 0
    o.x = encode_gathered(__byte_perm(x, 0, 0x1201u), lut);
    o.y = encode_gathered(__byte_perm(x, y, 0x4534u), lut);
    o.z = encode_gathered(__byte_perm(y, z, 0x3423u), lut);
    o.w = encode_gathered(__byte_perm(z, 0, 0x2312u), lut);
#else
    o.x = encode_v24<true>(__byte_perm(x, 0, 0x4012u), lut);
    o.y = encode_v24<false>(__byte_perm(x, y, 0x3345u), lut);
    o.z = encode_v24<false>(__byte_perm(y, z, 0x2234u), lut);
    o.w = encode_v24<true>(__byte_perm(z, 0, 0x4123u), lut);
#endif
    return o;
}

// A 4096-entry table of character pairs (12-bit index -> the characters of
// two adjacent 6-bit fields), built per block from the 64-entry alphabet
// (build_pairs): a triple, taken as the 24-bit number s1<<16 | s2<<8 | s3
// (Sec. 2), needs two 16-bit lookups instead of four 8-bit ones and fewer
// field extractions. Measured on 1 GiB: 2815 GB/s of input against 2746 with
// the 64-entry table (the random 12-bit indices cost some bank conflicts, but
// fewer ALU instructions).
__device__ __forceinline__ void build_pairs(uint16_t* pairs, const uint8_t* lut, int tid,
                                            int nthreads) {
    for (int i = tid; i < 4096; i += nthreads)
        pairs[i] = uint16_t(uint32_t(lut[i >> 6]) | (uint32_t(lut[i & 63]) << 8));
}
template <bool kClean>
__device__ __forceinline__ uint32_t encode_pairs(uint32_t v, const uint16_t* pairs) {
    const uint32_t hi = kClean ? v >> 12 : (v >> 12) & 0xFFFu;
    return __byte_perm(uint32_t(pairs[hi]), uint32_t(pairs[v & 0xFFFu]), 0x5410u);
}
__device__ __forceinline__ uint4 encode12_pairs(uint32_t x, uint32_t y, uint32_t z,
                                                const uint16_t* pairs) {
    uint4 o;
    o.x = encode_pairs<true>(__byte_perm(x, 0, 0x4012u), pairs);
    o.y = encode_pairs<false>(__byte_perm(x, y, 0x3345u), pairs);
    o.z = encode_pairs<false>(__byte_perm(y, z, 0x2234u), pairs);
    o.w = encode_pairs<true>(__byte_perm(z, 0, 0x4123u), pairs);
    return o;
}

// ------------------------------------------------------------------ decode step
// Sec. 2 / Sec. 3.2: four characters (little-endian word, first character in
// the low byte) -> the 24-bit value a<<18 | b<<12 | c<<6 | d, whose bytes
// from high to low are the three output bytes. `err` collects the OR of the
// translated values; bit 7 set means a byte outside the alphabet.
__device__ __forceinline__ uint32_t decode4(uint32_t w, const uint8_t* lut, uint32_t& err) {
    const uint32_t a = lut[__byte_perm(w, 0, 0x4440u)];
    const uint32_t b = lut[__byte_perm(w, 0, 0x4441u)];
    const uint32_t c = lut[__byte_perm(w, 0, 0x4442u)];
    const uint32_t d = lut[__byte_perm(w, 0, 0x4443u)];
    err |= a | b | c | d;
    return ((a * 64u + b) * 64u + c) * 64u + d;
}

// Packs four 24-bit values into 12 output bytes (three words), each value
// contributing its bytes from high to low.
__device__ __forceinline__ uint3 pack4x24(uint32_t q0, uint32_t q1, uint32_t q2, uint32_t q3) {
    uint3 o;
    o.x = __byte_perm(q0, q1, 0x6012u);
    o.y = __byte_perm(q1, q2, 0x5601u);
    o.z = __byte_perm(q2, q3, 0x4560u);
    return o;
}

// 16 bytes starting `off` bytes into a 4-byte aligned shared buffer (off a
// multiple of 4 plus `sh`, sh in 0..3), re-aligned with funnel shifts from
// five word loads. Reads up to 4 bytes past off + 16 when sh != 0.
__device__ __forceinline__ uint4 load16_shifted(const uint8_t* sbuf, uint32_t off, uint32_t sh) {
    const uint32_t* w = reinterpret_cast<const uint32_t*>(sbuf + (off & ~3u));
    const uint32_t w0 = w[0], w1 = w[1], w2 = w[2], w3 = w[3], w4 = sh ? w[4] : 0u;
    const uint32_t s = 8 * sh;
    return make_uint4(__funnelshift_r(w0, w1, s), __funnelshift_r(w1, w2, s),
                      __funnelshift_r(w2, w3, s), __funnelshift_r(w3, w4, s));
}

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the phase with the given parity to complete; false after
// kWaitLimitNs without completion.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (;;) {
        for (int i = 0; i < 16; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_timer_ns() - t0 > kWaitLimitNs) return false;
    }
}

// Bulk copy global -> shared; completion is signalled on `bar` as
// transaction bytes. Addresses 16-byte aligned, size a multiple of 16.
__device__ __forceinline__ void bulk_load(void* dst_smem, const void* src_gmem, uint32_t bytes,
                                          uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Bulk copy shared -> global in the current bulk group.
__device__ __forceinline__ void bulk_store(void* dst_gmem, const void* src_smem, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst_gmem),
                 "r"(smem_addr(src_smem)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() {
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// Waits until at most N committed bulk groups still read shared memory.
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}

// Waits until at most N committed bulk groups are still in flight.
template <int N>
__device__ __forceinline__ void bulk_wait_all() {
    asm volatile("cp.async.bulk.wait_group %0;" ::"n"(N) : "memory");
}

// Orders this thread's generic-proxy shared-memory writes before later
// async-proxy (bulk copy) reads of the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void st_global_cs(uint4* p, uint4 v) {
    asm volatile("st.global.cs.v4.u32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w)
                 : "memory");
}

// Minimum over the warp of a 64-bit value (only the full warp may call it).
__device__ __forceinline__ uint64_t warp_min_u64(uint64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u < v ? u : v;
    }
    return v;
}

}  // namespace b64
