// Shared-memory helpers of the batched and MIME kernels: re-alignment
// (strings and MIME documents start at any byte) and table lookups.
#pragma once

#include <cstdint>

namespace b64 {

// load16_shifted for off mod 16 the same in every lane (lanes 16 bytes
// apart): two aligned 128-bit loads, which keep the shared-memory
// accesses free of bank conflicts (five 32-bit loads 16 bytes apart would
// meet four lanes in a bank), then funnel shifts. Reads up to 32 bytes
// from off & ~15.
__device__ __forceinline__ uint4 load16_shifted_u(const uint8_t* sbuf, uint32_t off) {
    const uint32_t A = off & ~15u, r = off & 15u, sb = 8 * (r & 3u);
    const uint4 a = *reinterpret_cast<const uint4*>(sbuf + A);
    if (r == 0) return a;
    const uint4 b = *reinterpret_cast<const uint4*>(sbuf + A + 16);
    uint32_t v0, v1, v2, v3, v4;
    switch (r >> 2) {  // the same in every lane
        case 0: v0 = a.x; v1 = a.y; v2 = a.z; v3 = a.w; v4 = b.x; break;
        case 1: v0 = a.y; v1 = a.z; v2 = a.w; v3 = b.x; v4 = b.y; break;
        case 2: v0 = a.z; v1 = a.w; v2 = b.x; v3 = b.y; v4 = b.z; break;
        default: v0 = a.w; v1 = b.x; v2 = b.y; v3 = b.z; v4 = b.w; break;
    }
    return make_uint4(__funnelshift_r(v0, v1, sb), __funnelshift_r(v1, v2, sb),
                      __funnelshift_r(v2, v3, sb), __funnelshift_r(v3, v4, sb));
}

// decode4 for a 256-entry table at a 256-byte aligned shared-memory address
// `base`: the address of each character's entry is built by one byte permute
// (the character as its low byte, the table's upper address bytes above it)
// instead of an extract and an add. The four entries are OR-ed into err.
__device__ __forceinline__ uint32_t lds_u8(uint32_t addr) {
    uint32_t v;
    asm("ld.shared.u8 %0, [%1];" : "=r"(v) : "r"(addr));
    return v;
}
__device__ __forceinline__ uint32_t decode4_at(uint32_t w, uint32_t base, uint32_t& err) {
    const uint32_t a = lds_u8(__byte_perm(w, base, 0x7650u));
    const uint32_t b = lds_u8(__byte_perm(w, base, 0x7651u));
    const uint32_t c = lds_u8(__byte_perm(w, base, 0x7652u));
    const uint32_t d = lds_u8(__byte_perm(w, base, 0x7653u));
    err |= a | b | c | d;
    return ((a * 64u + b) * 64u + c) * 64u + d;
}

// Writes bytes 0 .. n-1 (n <= 16) of v (little-endian words) to q, which is
// 4-byte aligned: whole words, then a 16-bit and an 8-bit store for the rest.
__device__ __forceinline__ void store_head_aligned(uint8_t* q, uint4 v, uint32_t n) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (uint32_t k = 0; k < 4; ++k) {
        if (4 * k + 4 <= n) {
            reinterpret_cast<uint32_t*>(q)[k] = w[k];
        } else if (4 * k < n) {
            const uint32_t r = n - 4 * k;  // 1..3
            if (r >= 2) *reinterpret_cast<uint16_t*>(q + 4 * k) = uint16_t(w[k]);
            if (r & 1u) q[4 * k + (r & 2u)] = uint8_t(w[k] >> (8 * (r & 2u)));
        }
    }
}

}  // namespace b64
