// Counter-based Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11) and the transforms used by the kernels.
//
// Counter layout shared with the CPU oracle (which has its own implementation):
//   (path k, fine step q or inner index l, copy, stream << 24 | block)
// key = (seed low 32 bits, seed high 32 bits). Stream 1 feeds the outer-path
// normals (four per block), stream 2 the inner default clocks (four
// counterparties per block). copy is 0 for the simulation itself; a twin copy b
// of the twin Monte Carlo validation draws its outer normals after the branch date
// and all its inner clocks with copy = b.
#pragma once
#include <stdint.h>

namespace cva {

constexpr uint32_t kStreamOuter = 1u;
constexpr uint32_t kStreamInner = 2u;

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Uniform on (0,1): (m + 1/2) 2^-23 with m the top 23 bits; exact in binary32.
__device__ __forceinline__ float uniform23(uint32_t x)
{
    return (__uint2float_rn(x >> 9) + 0.5f) * 1.1920928955078125e-07f;
}

// Box-Muller on a pair of uniforms: (rad cos 2 pi u2, rad sin 2 pi u2).
__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, float &z0, float &z1)
{
    const float u1 = uniform23(a), u2 = uniform23(b);
    const float rad = sqrtf(-2.0f * logf(u1));
    float s, c;
    sincospif(2.0f * u2, &s, &c);
    z0 = rad * c;
    z1 = rad * s;
}

}  // namespace cva
