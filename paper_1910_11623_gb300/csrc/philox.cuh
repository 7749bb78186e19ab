// Device-side Philox4x32-10 and Box-Muller.
//
// Philox4x32-10 is the counter-based generator of Salmon, Moraes, Dror and
// Shaw, "Parallel Random Numbers: As Easy as 1, 2, 3" (SC'11), Section 4:
// each round multiplies counter words 0 and 2 by two fixed 32-bit constants,
// mixes the high halves with the other counter words and the key, and the key
// advances by two Weyl constants between rounds.  The paper being implemented
// only asks for Delta W_n ~ N(0, Delta t_n) (Section 2.2, Eq. "disc
// equations"); a counter-based generator makes every increment a pure function
// of (key, step, path, dimension, iteration), so the increments are never
// stored and can be regenerated anywhere.
#pragma once
#include <stdint.h>

namespace fbsde {

struct u32x4 { uint32_t x, y, z, w; };

__host__ __device__ __forceinline__ void philox_mulhilo(uint32_t a, uint32_t b, uint32_t& hi,
                                                         uint32_t& lo) {
#ifdef __CUDA_ARCH__
    hi = __umulhi(a, b);
    lo = a * b;
#else
    uint64_t p = (uint64_t)a * (uint64_t)b;
    hi = (uint32_t)(p >> 32);
    lo = (uint32_t)p;
#endif
}

// Ten rounds; the key is bumped before rounds 1..9.
__host__ __device__ __forceinline__ u32x4 philox4x32_10(u32x4 c, uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint32_t hi0, lo0, hi1, lo1;
        philox_mulhilo(M0, c.x, hi0, lo0);
        philox_mulhilo(M1, c.z, hi1, lo1);
        u32x4 n;
        n.x = hi1 ^ c.y ^ k0;
        n.y = lo1;
        n.z = hi0 ^ c.w ^ k1;
        n.w = lo0;
        c = n;
    }
    return c;
}

// u = (k + 1/2) 2^-32 in (0, 1).  In FP32 the conversion of k rounds to 24
// bits (relative error <= 2^-24), and u may round up to 1.0f for the top
// 2^7 words, where -2 ln u is then 0 instead of < 2^-24: both are below FP32
// resolution of the resulting normal's magnitude scale.
__device__ __forceinline__ float philox_uniform(uint32_t k) {
    return fmaf((float)k, 2.3283064365386963e-10f, 1.1641532182693481e-10f);
}

// Box-Muller (Box & Muller 1958): (u1, u2) -> sqrt(-2 ln u1) (cos, sin)(2 pi u2).
// Accurate CUDA library functions; sincospif avoids rounding 2 pi u2.
__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, float& z0, float& z1) {
    float u1 = philox_uniform(a), u2 = philox_uniform(b);
    float rad = sqrtf(-2.0f * logf(u1));
    float s, c;
    sincospif(2.0f * u2, &s, &c);
    z0 = rad * c;
    z1 = rad * s;
}

}  // namespace fbsde
