// Philox4x32-10 counter-based random numbers (Salmon, Moraes, Dror and
// Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC 2011): ten rounds
// of a multiply-xor bijection of a 128-bit counter under a 64-bit key that
// is bumped by fixed Weyl increments between rounds.  Written from that
// definition; compiles for the host too so the known-answer vectors of the
// published reference distribution can be checked without a GPU.
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define LBM_HD __host__ __device__ __forceinline__
#else
#define LBM_HD inline
#endif

namespace lbm {

LBM_HD uint32_t philox_mulhi(uint32_t a, uint32_t b) {
#if defined(__CUDA_ARCH__)
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
#endif
}

// c: the counter on entry, the four output words on return.
LBM_HD void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;   // round multipliers
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;   // key increments
#if defined(__CUDA_ARCH__)
#pragma unroll
#endif
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        const uint32_t hi0 = philox_mulhi(M0, c[0]), lo0 = M0 * c[0];
        const uint32_t hi1 = philox_mulhi(M1, c[2]), lo1 = M1 * c[2];
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

// Field j (0..8) of 13 random bits from a 128-bit block.
LBM_HD uint32_t bits13(const uint32_t w[4], int j) {
    const int off = 13 * j, q = off >> 5, s = off & 31;
    const uint64_t pair = (uint64_t)w[q] | ((uint64_t)(q < 3 ? w[q + 1] : 0u) << 32);
    return (uint32_t)(pair >> s) & 0x1fffu;
}

}  // namespace lbm
