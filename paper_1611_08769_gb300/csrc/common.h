// Shared definitions of the native library: parameters, wire references,
// gate descriptors (host compiler <-> device kernels), error reporting.
#pragma once

#include <cstdint>
#include <string>

#include "../../include/sfft.h"

namespace sfft {

// Error reporting: thread-local message, returned code.
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);

struct Shape {
  uint32_t n, ell, m, chi;
  uint32_t L;      // limbs per element (ell / 32)
  uint32_t NP1;    // elements per row (n + 1)
  uint32_t W;      // words per row (NP1 * L)
  uint32_t Ng;     // rows (= NP1 * ell)
  uint64_t ctw;    // words per ciphertext (Ng * W)
};

// Validates and expands parameters; returns SFFT_OK or an error code.
int make_shape(const sfft_params* p, Shape* s, bool need_square_key);

// ---------------------------------------------------------------------------
// Wire references inside gate descriptors.
//   bits 31..30  region: 0 scratch pool, 1 input buffer, 2 output buffer,
//                3 generated (encryption R matrix of ciphertext `slot`)
//   bits 29..0   slot (ciphertext index within the region)
// REF_NONE marks an absent output.
// ---------------------------------------------------------------------------
constexpr uint32_t REG_SCRATCH = 0, REG_IN = 1, REG_OUT = 2, REG_GEN = 3;
constexpr uint32_t REF_NONE = 0xFFFFFFFFu;
constexpr uint32_t SLOT_MASK = 0x3FFFFFFFu;
inline uint32_t make_ref(uint32_t region, uint32_t slot) { return (region << 30) | slot; }

// Gate descriptor: out = c0 P + c1 A + c2 B + c3 BitDecomp(A~) B, where A~ is
// A, or P - A when flag bit 0 is set. Codes pack (c0, c1, c2, c3) as signed
// nibbles: c0 | c1 << 4 | c2 << 8 | c3 << 12; code0 in bits 0..15, code1 in
// bits 16..31 of `code`.
struct alignas(16) GateDesc {
  uint32_t a, b, o0, o1;
};
struct GateAux {
  uint32_t code;   // code0 | code1 << 16
  uint32_t flags;  // bit 0: complement A before BitDecomp
};

inline uint16_t pack_code(int c0, int c1, int c2, int c3) {
  return (uint16_t)(((c0 & 15)) | ((c1 & 15) << 4) | ((c2 & 15) << 8) | ((c3 & 15) << 12));
}

// Code patch of a refresh program: gate `gate` takes a selected operand
// beta * C (beta a public bit of a refreshed ciphertext), so its coefficients
// become (c0, c1 bA, c2 bB, c3 bA bB) for both output codes of `code`. bA is
// bit a_pos % ell of element a_pos / ell of row ell - 1 of source ciphertext
// a_ct (1 when a_ct == REF_NONE); bB likewise.
struct PatchDesc {
  uint32_t gate, code, a_ct, a_pos, b_ct, b_pos, pad0, pad1;
};

// Output fix-up: materialises an output that is not written by a gate
// (an alias of another wire, a complemented wire, or a trivial constant).
//   kind 0: copy src; 1: P - src; 2: zero matrix; 3: P
struct FixDesc {
  uint32_t dst, src, kind, pad;
};

}  // namespace sfft
