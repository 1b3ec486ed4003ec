// rng.cuh -- the counter-based random numbers of the PIC step.
//
// SplitMix64 finaliser (Steele, Lea & Flood 2014) chained over four key
// words, h <- mix(h ^ word + gamma).  Injection keys are (seed, step,
// quadrangle, (j << 8) | slot); collision keys put 2^40 + cell in the third
// word (a quadrangle index never reaches 2^40) and the cell-order keys 2^41
// there, so the streams never meet.
#pragma once
#include <cstdint>

namespace pf {

constexpr uint64_t RNG_GAMMA = 0x9E3779B97F4A7C15ULL;
constexpr uint64_t RNG_COLL_DOMAIN = 1ULL << 40;
constexpr uint64_t RNG_SHUF_DOMAIN = 1ULL << 41;

__device__ __forceinline__ uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t hash4(uint64_t w0, uint64_t w1, uint64_t w2, uint64_t w3)
{
    uint64_t h = mix64((0ULL ^ w0) + RNG_GAMMA);
    h = mix64((h ^ w1) + RNG_GAMMA);
    h = mix64((h ^ w2) + RNG_GAMMA);
    return mix64((h ^ w3) + RNG_GAMMA);
}

// uniform in [0, 1): the top 53 bits of the chain over
// (seed, step, quad, (j << 8) | slot), times 2^-53
__device__ __forceinline__ double uniform01(uint64_t seed, uint64_t step, uint64_t quad,
                                            uint64_t j, uint64_t slot)
{
    return (double)(hash4(seed, step, quad, (j << 8) | (slot & 0xFF)) >> 11) * 0x1.0p-53;
}

}  // namespace pf
