// Shared-memory re-alignment shared by the batched kernels (strings and
// MIME documents start at any byte).
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

}  // namespace b64
