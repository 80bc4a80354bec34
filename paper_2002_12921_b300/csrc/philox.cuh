// Counter-based Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel
// random numbers: as easy as 1, 2, 3", Sec. 5), device side.
//
// Round r (0..9) takes the key (k0 + r W0, k1 + r W1) mod 2^32; those round
// keys are the same for every sample, so the host computes them once and the
// kernel reads them from the parameter bank (an operand of the xor, no register).
#pragma once

#include <stdint.h>

namespace vegas {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

// Host helper: the ten round keys of a 64-bit seed.
inline void philox_round_keys(uint64_t seed, uint32_t rk0[10], uint32_t rk1[10]) {
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        rk0[r] = k0;
        rk1[r] = k1;
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
}

#ifdef __CUDACC__
// Ten rounds on (c0, c1, c2, c3).  One round: the 64-bit products M0 c0 and
// M1 c2 split into high and low words; the new words are
// (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)).
__device__ __forceinline__ void philox4x32_10(uint32_t& c0, uint32_t& c1, uint32_t& c2,
                                              uint32_t& c3, const unsigned (&rk0)[10],
                                              const unsigned (&rk1)[10]) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(kPhiloxM0, c0);
        const uint32_t lo0 = kPhiloxM0 * c0;
        const uint32_t hi1 = __umulhi(kPhiloxM1, c2);
        const uint32_t lo1 = kPhiloxM1 * c2;
        c0 = hi1 ^ c1 ^ rk0[r];
        c1 = lo1;
        c2 = hi0 ^ c3 ^ rk1[r];
        c3 = lo0;
    }
}
#endif

}  // namespace vegas
