// Counter-based SplitMix64 streams (host and device).
//
// The paper does not specify its randomness; this library fixes it so that
// keys and ciphertexts are reproducible from seeds:
//   mix64      the SplitMix64 output finaliser (Steele, Lea, Flood 2014)
//   out(s, k)  = mix64(s + (k + 1) * 0x9E3779B97F4A7C15): k-th output of the
//              SplitMix64 generator started at state s
//   key(seed, d) = mix64(seed ^ d * 0xD1B54A32D192ED03), domains
//              1 secret t, 2 matrix B, 3 error e, 4 encryption matrices R
//   R of ciphertext c: stream out(key(enc_seed, 4), c), bits LSB first,
//              row-major over the Ng x m matrix.
#pragma once

#include <cstdint>

#if defined(__CUDACC__)
#define SFFT_HD __host__ __device__ __forceinline__
#else
#define SFFT_HD inline
#endif

namespace sfft {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kTagMul = 0xD1B54A32D192ED03ull;
constexpr uint32_t kDomT = 1, kDomB = 2, kDomE = 3, kDomR = 4;

SFFT_HD uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

SFFT_HD uint64_t stream_out(uint64_t state, uint64_t k) { return mix64(state + (k + 1) * kGamma); }

SFFT_HD uint64_t domain_key(uint64_t seed, uint32_t domain) {
  return mix64(seed ^ (uint64_t)domain * kTagMul);
}

SFFT_HD uint64_t ct_stream(uint64_t enc_seed, uint64_t ct_index) {
  return stream_out(domain_key(enc_seed, kDomR), ct_index);
}

// 32-bit word `w` of the R bit string of one ciphertext (word w holds bits
// 32w .. 32w+31 of the row-major Ng x m matrix).
SFFT_HD uint32_t r_word(uint64_t state, uint64_t w) {
  uint64_t v = stream_out(state, w >> 1);
  return (uint32_t)(v >> (32 * (w & 1)));
}

}  // namespace sfft
