// Counter-based uniforms on the device: SplitMix64 (Steele, Lea and Flood,
// "Fast splittable pseudorandom number generators", OOPSLA 2014) used as a
// counter-based generator.  For a seed, an event index i and a row k:
//   key = mix(seed),  z = mix(key + (64 i + k + 1) * 0x9E3779B97F4A7C15)
//   u   = ((z >> 11) + 0.5) * 2^-53   in the open interval (0, 1)
// with mix the SplitMix64 finaliser.  The value depends only on (seed, i, k),
// so any event of a batch can be drawn alone and ranks draw disjoint events.
#pragma once
#include <cstdint>

namespace mg {

constexpr int kRngRowStride = 64;   // counter slots per event
constexpr int kRngRowUnweight = 63;  // row of the unweighting uniform

__host__ __device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ double sm64_uniform(uint64_t key, int64_t event, int row) {
  const uint64_t ctr = (uint64_t)event * (uint64_t)kRngRowStride + (uint64_t)(row + 1);
  const uint64_t z = sm64_mix(key + ctr * 0x9E3779B97F4A7C15ull);
  return ((double)(z >> 11) + 0.5) * 0x1.0p-53;
}

}  // namespace mg
