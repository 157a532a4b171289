// Device kernels of the level evaluator (integer path).
//
// A level is a list of independent ciphertext products (Sec. 7: a NAND in
// GSW is an N x N matrix product; Sec. 4 composes every other gate from it).
// Each gate computes, on compressed ciphertexts,
//     out = c0 P + c1 A + c2 B + c3 BitDecomp(A~) B   (mod 2^ell, per element)
// with A~ = A or P - A. Row i of BitDecomp(A~) is simply the bit string of
// row i of A~, so the product is a masked sum of B's rows:
//     K[i][w] = sum_k bit_k(A~_i) * B[k][w]   (w = word column, no carries yet)
// accumulated exactly in 64-bit per 32-bit limb, then carried limb by limb
// inside each Z_q element (the top carry is dropped: mod q = 2^ell).
#pragma once

#include <cstdint>

#include "common.h"
#include "kargs.h"
#include "rng.h"

namespace sfft {


// The region base is selected with constant indices: indexing the parameter
// array with a runtime value would copy the kernel arguments to local memory.
__device__ __forceinline__ uint32_t* resolve(const KArgs& a, uint32_t ref) {
  const uint32_t r = ref >> 30;
  uint32_t* base = r == 0 ? a.base[0] : r == 1 ? a.base[1] : r == 2 ? a.base[2] : a.base[3];
  return base + (uint64_t)(ref & SLOT_MASK) * a.ctw;
}

// Limb `l` of element `j` of row `i` of the gadget matrix P.
__device__ __forceinline__ uint32_t p_word(uint32_t i, uint32_t j, uint32_t l, uint32_t ell) {
  return (j == i / ell && l == (i % ell) / 32) ? (1u << (i % 32)) : 0u;
}

__device__ __forceinline__ int nib(uint32_t code, int k) {
  return (int)((int32_t)(code << (28 - 4 * k)) >> 28);
}

// One warp per (gate, 32-row tile); lane = row. CC word columns at a time.
template <int CC>
__global__ void __launch_bounds__(256) k_gate_generic(KArgs a) {
  const uint32_t tiles = a.Ng / 32;
  const uint64_t task = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (task >= a.n * tiles) return;
  const uint64_t g = task / tiles;
  const uint32_t i = (uint32_t)(task % tiles) * 32 + (threadIdx.x & 31);
  const GateDesc d = a.desc[g];
  const GateAux x = a.aux[g];
  const bool gen = (d.a >> 30) == REG_GEN;
  const uint32_t* A = gen ? nullptr : resolve(a, d.a);
  const uint64_t gst = gen ? stream_out(a.gen_state, d.a & SLOT_MASK) : 0;
  const uint32_t* B = resolve(a, d.b);
  uint32_t* O0 = d.o0 == REF_NONE ? nullptr : resolve(a, d.o0);
  uint32_t* O1 = d.o1 == REF_NONE ? nullptr : resolve(a, d.o1);
  const bool comp = (x.flags & 1u) != 0;
  const uint32_t W = a.W, L = a.L;
  const uint32_t* Arow = A ? A + (uint64_t)i * W : nullptr;
  int64_t carry0 = 0, carry1 = 0;
  for (uint32_t c0 = 0; c0 < W; c0 += CC) {
    uint64_t acc[CC];
#pragma unroll
    for (int c = 0; c < CC; c++) acc[c] = 0;
    uint32_t borrow = 0;
    for (uint32_t kw = 0; kw < W; kw++) {
      uint32_t aw = gen ? r_word(gst, (uint64_t)i * W + kw) : __ldg(Arow + kw);
      if (comp) {  // (P - A) with a borrow chain inside each element
        const uint32_t l = kw % L;
        if (l == 0) borrow = 0;
        const uint32_t pw = p_word(i, kw / L, l, a.ell);
        const uint64_t v = (uint64_t)pw - aw - borrow;
        aw = (uint32_t)v;
        borrow = (uint32_t)(v >> 63);
      }
      const uint32_t* brow = B + (uint64_t)kw * 32 * W + c0;
#pragma unroll 4
      for (uint32_t b = 0; b < 32; b++) {
        const uint32_t m = 0u - ((aw >> b) & 1u);
        const uint32_t* br = brow + (uint64_t)b * W;
#pragma unroll
        for (int c = 0; c < CC; c++)
          if (c0 + c < W) acc[c] += (uint64_t)(__ldg(br + c) & m);
      }
    }
    // epilogue: linear terms and carries, limb by limb inside each element
    const uint32_t code0 = x.code & 0xFFFFu, code1 = x.code >> 16;
#pragma unroll
    for (int c = 0; c < CC; c++) {
      const uint32_t w = c0 + c;
      if (w >= W) break;
      const uint32_t l = w % L;
      if (l == 0) carry0 = carry1 = 0;
      const int64_t aw = A ? (int64_t)__ldg(Arow + w) : 0;
      const int64_t bw = (int64_t)__ldg(B + (uint64_t)i * W + w);
      const int64_t pw = (int64_t)p_word(i, w / L, l, a.ell);
      const int64_t k = (int64_t)acc[c];
      if (O0) {
        int64_t v = nib(code0, 3) * k + nib(code0, 1) * aw + nib(code0, 2) * bw +
                    nib(code0, 0) * pw + carry0;
        O0[(uint64_t)i * W + w] = (uint32_t)v;
        carry0 = v >> 32;
      }
      if (O1) {
        int64_t v = nib(code1, 3) * k + nib(code1, 1) * aw + nib(code1, 2) * bw +
                    nib(code1, 0) * pw + carry1;
        O1[(uint64_t)i * W + w] = (uint32_t)v;
        carry1 = v >> 32;
      }
    }
  }
}

// Output fix-ups: kind 0 copy, 1 P - src, 2 zero, 3 P. One block per fix-up,
// one thread per (row, element).
__global__ void k_fixup(const FixDesc* fix, uint64_t n, KArgs a) {
  const uint64_t f = blockIdx.x;
  if (f >= n) return;
  const FixDesc d = fix[f];
  uint32_t* dst = a.base[REG_OUT] + (uint64_t)d.dst * a.ctw;
  const uint32_t* src = (d.kind <= 1) ? resolve(a, d.src) : nullptr;
  const uint32_t NP1 = a.W / a.L;
  for (uint32_t t = threadIdx.x; t < a.Ng * NP1; t += blockDim.x) {
    const uint32_t i = t / NP1, j = t % NP1;
    uint32_t borrow = 0;
    for (uint32_t l = 0; l < a.L; l++) {
      const uint64_t off = (uint64_t)i * a.W + j * a.L + l;
      const uint32_t pw = p_word(i, j, l, a.ell);
      uint32_t v;
      if (d.kind == 0) {
        v = src[off];
      } else if (d.kind == 1) {
        const uint64_t r = (uint64_t)pw - src[off] - borrow;
        v = (uint32_t)r;
        borrow = (uint32_t)(r >> 63);
      } else if (d.kind == 2) {
        v = 0;
      } else {
        v = pw;
      }
      dst[off] = v;
    }
  }
}

// Linear gates (c3 = 0): out = c0 P + c1 A + c2 B, limb carries inside each
// element (mod 2^ell). Grid = gates x blocks over the Ng (n+1) (row, element)
// tasks; one thread per task walks the element's L limbs.
__global__ void k_linear(KArgs a, uint32_t blocks_per_gate) {
  const uint64_t g = blockIdx.x / blocks_per_gate;
  if (g >= a.n) return;
  const GateDesc d = a.desc[g];
  const uint32_t code = a.aux[g].code & 0xFFFFu;
  const int c0 = nib(code, 0), c1 = nib(code, 1), c2 = nib(code, 2);
  const uint32_t* A = resolve(a, d.a);
  const uint32_t* B = resolve(a, d.b);
  uint32_t* O = resolve(a, d.o0);
  const uint32_t NP1 = a.W / a.L;
  const uint32_t t = (blockIdx.x % blocks_per_gate) * blockDim.x + threadIdx.x;
  if (d.o0 == REF_NONE || t >= a.Ng * NP1) return;
  const uint32_t i = t / NP1, j = t % NP1;
  const uint64_t base = (uint64_t)i * a.W + j * a.L;
  int64_t carry = 0;
  for (uint32_t l = 0; l < a.L; l++) {
    const int64_t v = (int64_t)c0 * p_word(i, j, l, a.ell) + (int64_t)c1 * A[base + l] +
                      (int64_t)c2 * B[base + l] + carry;
    O[base + l] = (uint32_t)v;
    carry = v >> 32;
  }
}

// Code patches of a refresh program (PatchDesc), one thread per patch: each
// selector bit is read from row ell - 1 of its refreshed ciphertext in src.
__device__ __forceinline__ int src_bit(const uint32_t* src, uint64_t ctw, uint32_t row_word0,
                                       uint32_t L, uint32_t ell, uint32_t ct, uint32_t pos) {
  if (ct == REF_NONE) return 1;
  const uint32_t j = pos / ell, b = pos % ell;
  return (src[(uint64_t)ct * ctw + row_word0 + j * L + b / 32] >> (b % 32)) & 1;
}

__global__ void k_patch_codes(const PatchDesc* pd, uint64_t n, GateAux* aux, const uint32_t* src,
                              uint64_t ctw, uint32_t row_word0, uint32_t L, uint32_t ell) {
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const PatchDesc d = pd[t];
  const int ba = src_bit(src, ctw, row_word0, L, ell, d.a_ct, d.a_pos);
  const int bb = src_bit(src, ctw, row_word0, L, ell, d.b_ct, d.b_pos);
  uint32_t out = 0;
  for (int h = 0; h < 2; h++) {
    const uint32_t k = (d.code >> (16 * h)) & 0xFFFFu;
    const int c0 = nib(k, 0), c1 = nib(k, 1) * ba, c2 = nib(k, 2) * bb, c3 = nib(k, 3) * ba * bb;
    const uint32_t packed = (uint32_t)(c0 & 15) | ((uint32_t)(c1 & 15) << 4) |
                            ((uint32_t)(c2 & 15) << 8) | ((uint32_t)(c3 & 15) << 12);
    out |= packed << (16 * h);
  }
  aux[d.gate].code = out;
}

// Row ell-1 of each ciphertext (what decryption reads).
__global__ void k_gather_rows(const uint32_t* ct, uint64_t n, uint64_t ctw, uint32_t W,
                              uint32_t row, uint32_t* out) {
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * W) return;
  const uint64_t c = t / W;
  const uint32_t w = (uint32_t)(t % W);
  out[t] = ct[c * ctw + (uint64_t)row * W + w];
}

}  // namespace sfft
