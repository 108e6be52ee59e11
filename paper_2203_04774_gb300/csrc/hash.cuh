// The set hash of the device count + hash consumers (consumer.cu, noalloc.cu):
//   H = sum over triples of h(a, b, c) mod 2^64,
//   h(a, b, c) = mix(mix(mix(a + G) + b + G) + c + G),
// G = 0x9e3779b97f4a7c15, mix = the splitmix64 finaliser (Steele, Lea and
// Flood, OOPSLA 2014).  One definition for every consumer of the library.
#pragma once

#include <stdint.h>

namespace tl {

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t triple_hash(uint32_t a, uint32_t b, uint32_t c) {
  const uint64_t G = 0x9e3779b97f4a7c15ull;
  uint64_t v = mix64((uint64_t)a + G);
  v = mix64(v + (uint64_t)b + G);
  return mix64(v + (uint64_t)c + G);
}

}  // namespace tl
