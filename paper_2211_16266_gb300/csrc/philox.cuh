// Philox4x64-10 counter-based generator on the device.
//
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3"
// (SC'11): each round multiplies counter words 0 and 2 by two fixed 64-bit
// constants, mixes the high halves with words 1 and 3 and the round key, and
// the key advances by two Weyl constants per round. Counter and key layout
// of the densification: counter (v*W + u, iteration, stage, 0), key
// (seed, keyframe id); stage 0 draws the initial plane, stage 1+i the i-th
// refinement test.
#pragma once

#include <stdint.h>

namespace pmsp {

struct U4 {
    float x, y, z, w;
};

__device__ __forceinline__ void philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                              uint64_t k0, uint64_t k1, uint64_t out[4]) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
        const uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
        const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

// Four uniforms in [0, 1) from the top 24 bits of each word (exact in FP32).
__device__ __forceinline__ U4 draw_uniform4(uint64_t pixel, uint64_t iter, uint64_t stage, uint64_t seed,
                                            uint64_t key1) {
    uint64_t w[4];
    philox4x64_10(pixel, iter, stage, 0ull, seed, key1, w);
    const float s = 1.0f / 16777216.0f;
    U4 u;
    u.x = (float)(uint32_t)(w[0] >> 40) * s;
    u.y = (float)(uint32_t)(w[1] >> 40) * s;
    u.z = (float)(uint32_t)(w[2] >> 40) * s;
    u.w = (float)(uint32_t)(w[3] >> 40) * s;
    return u;
}

}  // namespace pmsp
