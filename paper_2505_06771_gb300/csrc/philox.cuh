// philox.cuh -- counter-based random numbers for the environment step (device side).
//
// Philox4x32-10 as defined by Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy
// as 1, 2, 3" (SC 2011): ten rounds, each two 32x32->64-bit products whose halves are mixed
// with the other counter words and the key; the key is bumped by two Weyl constants between
// rounds.  Counter = (env, episode, purpose << 24 | index, step or attempt), key = 64-bit seed.
#pragma once
#include <cstdint>

namespace rl {

struct Words4 {
    uint32_t w[4];
};

__device__ __forceinline__ Words4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t a_hi = __umulhi(0xD2511F53u, c0), a_lo = 0xD2511F53u * c0;
        const uint32_t b_hi = __umulhi(0xCD9E8D57u, c2), b_lo = 0xCD9E8D57u * c2;
        const uint32_t n0 = b_hi ^ c1 ^ k0;
        const uint32_t n2 = a_hi ^ c3 ^ k1;
        c0 = n0;
        c1 = b_lo;
        c2 = n2;
        c3 = a_lo;
    }
    Words4 r;
    r.w[0] = c0; r.w[1] = c1; r.w[2] = c2; r.w[3] = c3;
    return r;
}

// Draw purposes (the third counter word's top byte).
enum : uint32_t { kNoise = 1, kPos = 2, kGoal = 3, kNear = 4, kLevel = 5, kRes = 6, kNRes = 7 };

__device__ __forceinline__ Words4 draw(uint64_t seed, int env, int episode, uint32_t purpose,
                                       int index, uint32_t step) {
    return philox4x32_10((uint32_t)env, (uint32_t)episode, (purpose << 24) | (uint32_t)index,
                         step, (uint32_t)seed, (uint32_t)(seed >> 32));
}

// Uniform in [0, 1) on the 2^-24 grid: exact in binary32.
__device__ __forceinline__ float unit24(uint32_t w) {
    return __fmul_rn(__uint2float_rn(w >> 8), 5.9604644775390625e-08f);
}

// floor(w * k / 2^32), an integer in [0, k).
__device__ __forceinline__ int below(uint32_t w, uint32_t k) {
    return (int)(((uint64_t)w * (uint64_t)k) >> 32);
}

}  // namespace rl
