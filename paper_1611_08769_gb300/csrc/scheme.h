// Host-side helpers shared between the C ABI translation units.
#pragma once

#include <cstdint>
#include <vector>

namespace sfft {

// Fixed-point encoding of a signal (Sec. 4; Sec. 5 truncation):
// raw = floor(x * 2^f) mod 2^F, bit b of sample k part p at (2k + p) F + b.
void encode_signal(const double* re, const double* im, uint64_t count, uint32_t F, uint32_t f,
                   std::vector<uint8_t>* bits);

}  // namespace sfft
