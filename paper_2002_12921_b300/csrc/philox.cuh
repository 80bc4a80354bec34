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
// Rounds R0 .. R1-1 on (c0, c1, c2, c3).  One round: the 64-bit products M0 c0
// and M1 c2 split into high and low words; the new words are
// (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)).
template <int R0, int R1>
__device__ __forceinline__ void philox_rounds(uint32_t& c0, uint32_t& c1, uint32_t& c2,
                                              uint32_t& c3, const unsigned (&rk0)[10],
                                              const unsigned (&rk1)[10]) {
#pragma unroll
    for (int r = R0; r < R1; ++r) {
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

// All ten rounds.
__device__ __forceinline__ void philox4x32_10(uint32_t& c0, uint32_t& c1, uint32_t& c2,
                                              uint32_t& c3, const unsigned (&rk0)[10],
                                              const unsigned (&rk1)[10]) {
    philox_rounds<0, 10>(c0, c1, c2, c3, rk0, rk1);
}

// The calls of one sample share their first two rounds' work.  For the counter
// (i_lo, i_hi, Q_q, t) of call q, round 0 gives
//   (hi(M1 Q_q) ^ i_hi ^ k0_0, lo(M1 Q_q), hi(M0 i_lo) ^ t ^ k1_0, lo(M0 i_lo)):
// its words 2 and 3 do not depend on q, and words 0 and 1 do not depend on the
// sample.  Round 1 multiplies word 2 (the same for every call) and word 0 (the
// same for every sample of one i_hi).  So per sample only M0 i_lo and M1 times
// round-0 word 2 are needed, whatever the number of calls; the per-call
// constants below hold the rest.  The words are those of philox4x32_10.
struct PhiloxCallConst {
    uint32_t a;   // lo(M1 Q_q) ^ k0_1          -> round-1 word 0 = hi(M1 w2) ^ a
    uint32_t b;   // hi(M0 w0_q) ^ k1_1         -> round-1 word 2 = lo(M0 i_lo) ^ b
    uint32_t c;   // lo(M0 w0_q)                -> round-1 word 3
};

// Per-call constants for counter word 2 = q_word and sample-index high word i_hi.
__device__ __forceinline__ PhiloxCallConst philox_call_const(uint32_t q_word, uint32_t i_hi,
                                                             const unsigned (&rk0)[10],
                                                             const unsigned (&rk1)[10]) {
    const uint32_t w0 = __umulhi(kPhiloxM1, q_word) ^ i_hi ^ rk0[0];
    PhiloxCallConst k;
    k.a = (kPhiloxM1 * q_word) ^ rk0[1];
    k.b = __umulhi(kPhiloxM0, w0) ^ rk1[1];
    k.c = kPhiloxM0 * w0;
    return k;
}
#endif

}  // namespace vegas
