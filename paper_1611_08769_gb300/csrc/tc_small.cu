// Gate product for small ciphertexts (64 <= Ng <= 256) on the tensor cores.
//
// The GSW product K = BitDecomp(A~) B' (Sec. 7: an N x N matrix product per
// gate) is a {0,1} matrix times the entries of B'. For Ng <= 256 a whole
// gate fits in one CTA: A~ and B' (Ng^2 / 8 bytes each, 8 KB at n = 1,
// ell = 128) and the tensor-core image of B' stay in shared memory, and the
// gate's one or two 128-row output tiles are multiplied back to back, so B' is
// converted once per gate inside the kernel (no separate expansion pass)
// and nothing but the operands and the outputs crosses HBM.
//
// Arithmetic. Every ell-bit entry of B' is cut into 8-bit digits d; per
// output row i and digit column (element e, digit t)
//     S[i][e,t] = sum_k bit_k(A~_i) d_t(B'_k[e])  <=  Ng * 255  <  2^16.
// The MMA runs kind::f16 (fp16 x fp16 -> fp32). The A operand is the bits
// themselves, masked in place: a 32-bit word of A~ becomes 16 fp16 pairs,
// pair c holding bits c and c + 16 at one bit position p(c) in 10..14 of
// each half (the word, or a copy shifted by 5, 10 or -1 bits, AND a mask),
// so a set bit is the fp16 number with the single exponent bit p - 10 set:
// 2^-14, 2^-13, 2^-11, 2^-7 or 2 for p = 10..14. The B operand carries the
// matching factor, d * 2^-6 / value(p) (2^8, 2^7, 2^5, 2^1, 2^-7), so every
// product is d * 2^-6 exactly and the fp32 accumulator holds S * 2^-6, a
// multiple of 2^-6 below 2^10: exact. The K order is the same permutation on
// both sides (K position 32 w + 2 c + h is bit 32 w + c + 16 h of the row).
// Every accumulator starts at 2^17 (its ulp is 2^-6), so its bits after the
// MMAs are those of 2^17 plus the integer S; the epilogue forms each 32-bit
// word of K from four such digit sums and adds c0 P + c1 A + c2 B with the
// element's limb carries, as the integer kernel does (half adders and ORs,
// the codes the circuits mostly use, by shorter dedicated carry chains).
//
// Roles (one persistent CTA of 18 warps per SM, 19 in the persistent form;
// CTA b takes the gates b, b + grid, ..., or in the persistent form claims
// chunks of gates in program order; a gate is one or two 128-row items):
//   warp 0       MMA issuer: per item Ng / 16 tcgen05.mma (M 128, N the digit
//                columns, K 16) from the A stage in tensor memory and the B
//                image in shared memory, then commits
//   warp 1       producer: bulk copies of A' and B' of each gate into a ring
//                slot of shared memory
//   warps 2, 3, 16, 17  B converters (one per SM sub-partition): B' -> its
//                128B-swizzled K-major fp16 image
//   warps 4..7   A expanders, one per tensor-memory lane quarter: thread =
//                row; complement (P - A) in registers when the gate asks for
//                it, mask the bits, store them to the item's A stage
//   warps 8..15  epilogue: accumulators -> output words, written in place
//                over the slot's A' and B' rows; the gate's outputs then leave
//                by two bulk stores (lane 0 of warp 8). In the persistent form
//                the outputs go straight to their global rows and
//   warp 18      (persistent form) publishes each finished gate: one
//                gpu-scope fence, the gate's done flag and its level's count,
//                off the epilogue's path
// Every wait is bounded (about 2 s); on timeout the kernel records
// KERR_MMA_TIMEOUT, drains its own MMAs and bulk stores, frees its tensor
// memory and returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>
#include <vector>

#include "common.h"
#include "kargs.h"
#include "plan.h"
#include "ptx.cuh"

namespace sfft {

namespace {

constexpr int kSmThreads = 576;                  // 18 warps
constexpr int kSmThreadsPersist = 608;           // + the publishing warp
constexpr uint32_t kSmTmemCols = 512;
constexpr uint32_t kSmMaxSlots = 8, kSmMaxAStages = 4, kSmMaxAcc = 8;
constexpr uint32_t kSmConvWarps = 4, kSmConvThreads = 128;   // warps 2, 3, 16, 17
constexpr uint32_t kSmExpWarp0 = 4, kSmEpiWarp0 = 8, kSmEpiWarps = 8, kSmPubWarp = 18;
constexpr uint32_t kSmBars = 64;                 // mbarrier slots (8 bytes each)
constexpr uint32_t kClaim = 4;                   // gates per claim of the persistent launch
constexpr uint32_t kSmMaxSmem = 232448;          // 227 KB opt-in per CTA

// Bounded wait on every lane of the warp; true on every lane iff all saw the
// phase complete.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* flag) {
  return __all_sync(0xFFFFFFFFu, mbar_wait_flag(bar, parity, flag));
}

// Four K=16 steps of one 64-wide atom: D (+)= A[at .. at + 31] * B^T, B's
// descriptor advancing 32 bytes (2 units) per step, A 8 columns per step;
// issued by one elected lane (the whole warp executes the statement).
__device__ __forceinline__ void mma_atom4(uint32_t d, uint32_t at, uint64_t b, uint32_t idesc,
                                          uint32_t acc) {
  asm volatile(
      "{\n .reg .pred e, p, t;\n .reg .b32 a1, a2, a3;\n .reg .b64 b1, b2, b3;\n"
      " elect.sync _|e, 0xffffffff;\n"
      " setp.ne.b32 p, %4, 0;\n setp.eq.b32 t, %4, %4;\n"
      " add.u32 a1, %1, 8;\n add.u32 a2, %1, 16;\n add.u32 a3, %1, 24;\n"
      " add.u64 b1, %2, 2;\n add.u64 b2, %2, 4;\n add.u64 b3, %2, 6;\n"
      " @e tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n"
      " @e tcgen05.mma.cta_group::1.kind::f16 [%0], [a1], b1, %3, t;\n"
      " @e tcgen05.mma.cta_group::1.kind::f16 [%0], [a2], b2, %3, t;\n"
      " @e tcgen05.mma.cta_group::1.kind::f16 [%0], [a3], b3, %3, t;\n}\n" ::"r"(d),
      "r"(at), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// One K=16 step (the last steps of an atom that is not full).
__device__ __forceinline__ void mma_one(uint32_t d, uint32_t at, uint64_t b, uint32_t idesc,
                                        uint32_t acc) {
  asm volatile(
      "{\n .reg .pred e, p;\n elect.sync _|e, 0xffffffff;\n setp.ne.b32 p, %4, 0;\n"
      " @e tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
      "r"(at), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void tmem_st_x16(uint32_t taddr, const uint32_t* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
      "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
      : "memory");
}

__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Bulk copy shared -> global (bulk-group completion).
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
               "r"(smem_u32(src)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// 32 bits of a row of A~ -> 16 fp16 pairs (K positions 2c, 2c + 1 <- bits c,
// c + 16), each set bit at position p(c) of its half: p = c + 10 for c < 5,
// c + 5 for c < 10, c for c < 15, 14 for c = 15.
__device__ __forceinline__ void bits_to_pairs(uint32_t x, uint32_t* v) {
  const uint32_t y10 = x << 10, y5 = x << 5, y1 = x >> 1;
#pragma unroll
  for (int c = 0; c < 5; c++) v[c] = y10 & (0x00010001u << (c + 10));
#pragma unroll
  for (int c = 5; c < 10; c++) v[c] = y5 & (0x00010001u << (c + 5));
#pragma unroll
  for (int c = 10; c < 15; c++) v[c] = x & (0x00010001u << c);
  v[15] = y1 & 0x40004000u;
}

// fp16 pair factor of the B operand for pair c: 2^-6 / value(p(c)), with
// value(p) = 2^(2^(p - 10) - 15): 2^8, 2^7, 2^5, 2^1, 2^-7 for p = 10..14.
__device__ __forceinline__ uint32_t b_factor(uint32_t c) {
  const uint32_t p = c < 5 ? c + 10 : c < 10 ? c + 5 : c < 15 ? c : 14u;
  const uint32_t h = p == 10 ? 0x5C00u : p == 11 ? 0x5800u : p == 12 ? 0x5000u : p == 13 ? 0x4000u : 0x2000u;
  return h | (h << 16);
}

__device__ __forceinline__ uint32_t hsub2(uint32_t a, uint32_t b) {
  uint32_t r;
  asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}

__device__ __forceinline__ uint32_t hmul2(uint32_t a, uint32_t b) {
  uint32_t r;
  asm("mul.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}

}  // namespace

struct SmShape {
  uint32_t mt;          // 128-row items per gate
  uint32_t ksteps;      // K = 16 MMA steps per item (Ng / 16)
  uint32_t atoms;       // 64-wide K atoms of the B image
  uint32_t dig;         // 8-bit digits per element (ell / 8)
  uint32_t ncols;       // MMA N: (n + 1) dig rounded up to 16
  uint32_t img_bytes;   // B image: atoms x ncols rows x 128 bytes
  uint32_t raw_bytes;   // one ciphertext: Ng W 4
  uint32_t slot_bytes;  // image + A' + B', 1024-byte multiple
  uint32_t nslots, nastages, nacc;
  uint32_t acols;       // tensor-memory columns of an A stage (Ng / 2)
  uint32_t acc0;        // first tensor-memory column of the A stages
  uint32_t smem_bytes;
};


// Slot metadata: the gate's descriptor, written by the producer with its
// bulk copies (visible to every role once raw_full completes).
struct SlotMeta {
  uint32_t a, b, o0, o1, code, flags, kind, gate;   // gate kNoGate: no more gates (persistent form)
};
constexpr uint32_t kNoGate = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Persistent launch: waits (bounded, ~2 s, also ending once `flag` is set)
// until *p >= target, with acquire semantics.
__device__ __forceinline__ bool wait_at_least32(const uint32_t* p, uint32_t target, volatile int* flag) {
  if (ld_acquire_u32(p) >= target) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0; it < kSpinLimit; it++) {
    __nanosleep(64);
    if (ld_acquire_u32(p) >= target) return true;
    if ((it & 63u) == 63u && (*flag || global_ns() - t0 > kWaitNs)) return false;
  }
  return false;
}

__device__ __forceinline__ bool wait_at_least64(const unsigned long long* p, unsigned long long target,
                                                volatile int* flag) {
  if (ld_acquire_u64(p) >= target) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0; it < kSpinLimit; it++) {
    __nanosleep(64);
    if (ld_acquire_u64(p) >= target) return true;
    if ((it & 63u) == 63u && (*flag || global_ns() - t0 > kWaitNs)) return false;
  }
  return false;
}

// Gate kinds with a specialised epilogue (codes as stored, after the
// compiler absorbed complemented operands): a half adder (output 0 XOR =
// A + B - 2K, output 1 AND = K), an OR (A + B - K); every other code runs the
// general form.
constexpr uint32_t kKindGeneric = 0, kKindHA = 1, kKindOR = 2;
constexpr uint32_t kCodeXOR = 0xE110u, kCodeAND = 0x1000u, kCodeOR = 0xF110u;

// Every accumulator starts at 2^17 (fp32 bits 0x48000000) instead of 0, so
// that its bits after the MMAs are 0x48000000 + S for a digit sum S (S 2^-6
// < 2^17 keeps the ulp at 2^-6): K words are assembled from the raw bits and
// the bias of the four digits of a word, 0x48000000 (1 + 2^16) after the
// byte shifts (the 2^8 and 2^24 copies wrap out of 32 bits), leaves once.
constexpr uint32_t kAccBiasBits = 0x48000000u;
constexpr uint64_t kWordBias = 0x480048000000ull;

__device__ __forceinline__ void tmem_st_x4(uint32_t taddr, uint32_t v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%1,%1,%1};" ::"r"(taddr), "r"(v) : "memory");
}

// Rows of LL-limb elements: aligned vector access where the limb count
// allows (16-byte for 4 limbs, 8-byte for 2), word by word otherwise.
template <int LL>
__device__ __forceinline__ void ld_elem(const uint32_t* p, uint32_t (&v)[LL]) {
  if constexpr (LL == 4) {
    const uint4 q = *reinterpret_cast<const uint4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else if constexpr (LL == 2) {
    const uint2 q = *reinterpret_cast<const uint2*>(p);
    v[0] = q.x; v[1] = q.y;
  } else {
#pragma unroll
    for (int k = 0; k < LL; k++) v[k] = p[k];
  }
}

template <int LL>
__device__ __forceinline__ void st_elem(uint32_t* p, const uint32_t (&v)[LL]) {
  if constexpr (LL == 4) {
    *reinterpret_cast<uint4*>(p) = make_uint4(v[0], v[1], v[2], v[3]);
  } else if constexpr (LL == 2) {
    *reinterpret_cast<uint2*>(p) = make_uint2(v[0], v[1]);
  } else {
#pragma unroll
    for (int k = 0; k < LL; k++) p[k] = v[k];
  }
}

// One element of LL words to a global row (explicit global stores; the
// shared-memory rows go through st_elem).
template <int LL>
__device__ __forceinline__ void st_elem_global(uint32_t* p, const uint32_t (&v)[LL]) {
  if constexpr (LL == 4) {
    asm volatile("st.global.v4.u32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3])
                 : "memory");
  } else if constexpr (LL == 2) {
    asm volatile("st.global.v2.u32 [%0], {%1, %2};" ::"l"(p), "r"(v[0]), "r"(v[1]) : "memory");
  } else {
#pragma unroll
    for (int k = 0; k < LL; k++) asm volatile("st.global.u32 [%0], %1;" ::"l"(p + k), "r"(v[k]) : "memory");
  }
}

// A row of W <= 8 words into registers (16-byte loads when W is a multiple of 4).
__device__ __forceinline__ void ld_row(const uint32_t* row, uint32_t W, uint32_t (&x)[8]) {
  if ((W & 3u) == 0) {
#pragma unroll
    for (uint32_t w = 0; w < 8; w += 4) {
      if (w < W) {
        const uint4 q = *reinterpret_cast<const uint4*>(row + w);
        x[w] = q.x; x[w + 1] = q.y; x[w + 2] = q.z; x[w + 3] = q.w;
      } else {
        x[w] = x[w + 1] = x[w + 2] = x[w + 3] = 0u;
      }
    }
  } else {
#pragma unroll
    for (uint32_t w = 0; w < 8; w++) x[w] = w < W ? row[w] : 0u;
  }
}

// ---------------------------------------------------------------------------
// Shared memory (from a 1024-aligned base):
//   nslots x slot     [B image | A' rows | B' rows]; the epilogue writes the
//                     outputs over A' (output 0) and B' (output 1)
//   slot metadata, mbarriers, the tensor-memory address slot, the stop flag
// Tensor memory (512 columns): nacc accumulators of ncols columns, then
// nastages A stages of Ng / 2 columns (row i in lane i % 128).
// Barriers (per ring slot s / A stage / accumulator):
//   raw_full[s]   the gate's A' and B' landed (producer's transaction count)
//   img_full[s]   the B image is written (four converter warps)
//   epi_done[s]   every epilogue warp wrote its outputs for the gate
//   slot_free[s]  the gate's outputs left the slot (bulk stores read it;
//                 lane 0 of warp 8 arrives), or were published (persistent
//                 form; the publishing warp arrives)
//   afull[a]      an item's A stage is written (four expander warps)
//   afree[a]      the item's MMAs are done (commit)
//   accfull[c]    an item's MMAs are done (commit)
//   accfree[c]    the epilogue read the accumulator (eight warps)
// Warps: 0 issuer, 1 producer, 2 3 16 17 converters (one per SM
// sub-partition), 4..7 expanders, 8..15 epilogue, 18 publisher (persistent
// form). The level form knows its gate count; the persistent form's roles
// stop at an end marker in the ring.
// ---------------------------------------------------------------------------
template <int LL, bool PERSIST>
__global__ void __launch_bounds__(PERSIST ? kSmThreadsPersist : kSmThreads, 1) k_gate_sm(KArgs a, SmShape t) {
  constexpr uint32_t kEll = 32u * LL, kDig = 4u * LL;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  SlotMeta* meta = (SlotMeta*)(smem + t.nslots * t.slot_bytes);
  uint64_t* bars = (uint64_t*)(meta + kSmMaxSlots);
  uint64_t* raw_full = bars;
  uint64_t* img_full = bars + 8;
  uint64_t* epi_done = bars + 16;
  uint64_t* slot_free = bars + 24;
  uint64_t* afull = bars + 32;
  uint64_t* afree = bars + 36;
  uint64_t* accfull = bars + 40;
  uint64_t* accfree = bars + 48;
  uint64_t* drain = bars + 56;
  uint32_t* tslot = (uint32_t*)(bars + 60);
  volatile int* sflag = (volatile int*)(tslot + 1);

  const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint64_t ngates = a.n;
  if (blockIdx.x >= ngates) return;
  constexpr bool persist = PERSIST;   // one launch across levels
  const uint32_t nloc = persist ? 0u : (uint32_t)((ngates - 1 - blockIdx.x) / gridDim.x + 1);
  const uint32_t items = nloc * t.mt;
  const uint32_t W = a.W, Ng = a.Ng, NP1 = W / LL;
  auto img_of = [&](uint32_t s) { return smem + s * t.slot_bytes; };
  auto araw_of = [&](uint32_t s) { return (uint32_t*)(smem + s * t.slot_bytes + t.img_bytes); };
  auto braw_of = [&](uint32_t s) {
    return (uint32_t*)(smem + s * t.slot_bytes + t.img_bytes + t.raw_bytes);
  };

  if (tid == 0) {
    for (uint32_t b = 0; b < kSmMaxSlots; b++) {
      mbar_init(&raw_full[b], 1u);
      mbar_init(&img_full[b], kSmConvWarps);
      mbar_init(&epi_done[b], kSmEpiWarps);
      mbar_init(&slot_free[b], 1u);
      mbar_init(&accfull[b], 1u);
      mbar_init(&accfree[b], kSmEpiWarps);
    }
    for (uint32_t b = 0; b < kSmMaxAStages; b++) {
      mbar_init(&afull[b], 4u);
      mbar_init(&afree[b], 1u);
    }
    mbar_init(drain, 1u);
    *sflag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(tslot, kSmTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    // ------------------------------------------------------------ MMA issuer
    const uint32_t idesc = idesc_f16(128, t.ncols);
    const uint32_t atom_units = (t.ncols * 128u) >> 4;   // descriptor units between atoms
    bool ok = true;
    uint32_t j = 0, m = 0, st = 0, stph = 0, acc = 0, accph = 0;
    for (uint32_t it = 0;; it++) {
      if (!persist && it >= items) break;
      const uint32_t s = j % t.nslots;
      if (persist && m == 0) {   // a gate's image (the end marker's slot is released too)
        if (!warp_wait(&img_full[s], (j / t.nslots) & 1u, sflag)) { ok = false; break; }
        if (meta[s].gate == kNoGate) break;
      }
      if (!warp_wait(&accfree[acc], accph, sflag)) { ok = false; break; }
      if (!warp_wait(&afull[st], stph, sflag)) { ok = false; break; }
      if (!persist && m == 0 && !warp_wait(&img_full[s], (j / t.nslots) & 1u, sflag)) { ok = false; break; }
      tc_fence_after();
      const uint32_t d = tmem + acc * t.ncols;
      const uint32_t at = tmem + t.acc0 + st * t.acols;
      const uint64_t b0 = sw128_desc(smem_u32(img_of(s)));
      uint32_t k = 0;
      for (uint32_t atom = 0; atom < t.atoms; atom++) {
        const uint64_t bd = b0 + (uint64_t)atom * atom_units;
        if (k + 4 <= t.ksteps) {
          mma_atom4(d, at + 8u * k, bd, idesc, 1u);
          k += 4;
        } else {
          for (uint32_t q = 0; k < t.ksteps; q++, k++) mma_one(d, at + 8u * k, bd + 2u * q, idesc, 1u);
        }
      }
      mma_commit_elected(&afree[st]);
      mma_commit_elected(&accfull[acc]);
      if (++st == t.nastages) { st = 0; stph ^= 1u; }
      if (++acc == t.nacc) { acc = 0; accph ^= 1u; }
      if (++m == t.mt) { m = 0; j++; }
    }
    if (!ok && lane == 0) *sflag = 1;
    mma_commit_elected(drain);   // tracks every MMA issued

  } else if (warp == 1) {
    // -------------------------------------------------------------- producer
    // a gate into ring slot s: its descriptor to the slot's metadata, its two
    // operands by bulk copies completing on raw_full[s]
    auto load_gate = [&](uint32_t s, uint64_t g, const GateDesc& gd, const GateAux& ax) {
      SlotMeta md;
      md.a = gd.a; md.b = gd.b; md.o0 = gd.o0; md.o1 = gd.o1;
      md.code = ax.code; md.flags = ax.flags;
      const uint32_t c0 = ax.code & 0xFFFFu, c1 = ax.code >> 16;
      md.kind = (c0 == kCodeXOR && c1 == kCodeAND) ? kKindHA
                : (c0 == kCodeOR && gd.o1 == REF_NONE) ? kKindOR : kKindGeneric;
      md.gate = (uint32_t)g;
      meta[s] = md;   // published by the arrival below (release)
      mbar_expect_tx(&raw_full[s], 2u * t.raw_bytes);
      bulk_g2s(araw_of(s), ct_ptr(a, gd.a), t.raw_bytes, &raw_full[s]);
      bulk_g2s(braw_of(s), ct_ptr(a, gd.b), t.raw_bytes, &raw_full[s]);
    };
    auto end_marker = [&](uint32_t s) {   // the other roles stop at this slot
      meta[s].gate = kNoGate;
      mbar_arrive(&raw_full[s]);
    };
    bool ok = true;
    if constexpr (!persist) {
      // gates b, b + grid, b + 2 grid, ... (one lane)
      if (lane == 0) {
        for (uint32_t j = 0; j < nloc; j++) {
          const uint32_t s = j % t.nslots, use = j / t.nslots;
          if (use && !mbar_wait_flag(&slot_free[s], (use - 1) & 1u, sflag)) { ok = false; break; }
          const uint64_t g = blockIdx.x + (uint64_t)j * gridDim.x;
          load_gate(s, g, a.desc[g], a.aux[g]);
        }
      }
    } else {
      // chunks of kClaim consecutive gates claimed in program order; lane k
      // fetches gate k's descriptor and checks its readiness, all lanes at
      // once; the gates are loaded in order, waiting (bounded) only for one
      // whose operands' producers, or whose level two up, were not done yet
      const uint32_t ep = *a.epoch;
      uint32_t j = 0;
      bool done = false;
      while (ok && !done) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(a.claim, kClaim);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        const uint64_t gk = (uint64_t)base + lane;
        const bool mine = lane < kClaim && gk < ngates;
        GateDesc gd{0, 0, REF_NONE, REF_NONE};
        GateAux ax{0, 0};
        uint32_t lev = 0;
        GateDeps dep{kNoGate, kNoGate};
        bool ready = true;
        if (mine) {
          gd = a.desc[gk];
          ax = a.aux[gk];
          lev = a.glev[gk];
          dep = a.gdep[gk];
          const uint32_t need = lev >= 2 ? a.lwidth[lev - 2] : 0u;
          ready = (lev < 2 || ld_acquire_u64(&a.ldone[lev - 2]) >= need) &&
                  (dep.a == kNoGate || ld_acquire_u32(&a.gflag[dep.a]) >= ep) &&
                  (dep.b == kNoGate || ld_acquire_u32(&a.gflag[dep.b]) >= ep);
        }
        for (uint32_t k = 0; k < kClaim; k++) {
          const uint32_t s = j % t.nslots, use = j / t.nslots;
          bool sok = true;
          if (lane == 0 && use) sok = mbar_wait_flag(&slot_free[s], (use - 1) & 1u, sflag);
          if (!__shfl_sync(0xFFFFFFFFu, (int)sok, 0)) { ok = false; break; }
          const uint64_t g = (uint64_t)base + k;
          if (g >= ngates) {
            if (lane == 0) end_marker(s);
            done = true;
            break;
          }
          bool dok = true;
          if (lane == k && !ready)
            dok = (lev < 2 || wait_at_least64(&a.ldone[lev - 2], a.lwidth[lev - 2], sflag)) &&
                  (dep.a == kNoGate || wait_at_least32(&a.gflag[dep.a], ep, sflag)) &&
                  (dep.b == kNoGate || wait_at_least32(&a.gflag[dep.b], ep, sflag));
          if (!__shfl_sync(0xFFFFFFFFu, (int)dok, k)) { ok = false; break; }
          GateDesc d;
          d.a = __shfl_sync(0xFFFFFFFFu, gd.a, k);
          d.b = __shfl_sync(0xFFFFFFFFu, gd.b, k);
          d.o0 = __shfl_sync(0xFFFFFFFFu, gd.o0, k);
          d.o1 = __shfl_sync(0xFFFFFFFFu, gd.o1, k);
          GateAux x;
          x.code = __shfl_sync(0xFFFFFFFFu, ax.code, k);
          x.flags = __shfl_sync(0xFFFFFFFFu, ax.flags, k);
          __syncwarp();   // lane k's acquire before lane 0's loads
          if (lane == 0) {
            asm volatile("fence.proxy.async.global;" ::: "memory");   // before the bulk loads read them
            load_gate(s, g, d, x);
          }
          j++;
        }
      }
    }
    if (!ok && lane == 0) *sflag = 1;

  } else if (warp == 2 || warp == 3 || warp == 16 || warp == 17) {
    // ----------------------------------------------------------- B converters
    // pair P = 16 w + c: rows k0 = 32 w + c and k0 + 16 of B' -> K positions
    // 2P, 2P + 1 of every digit row n = e dig + t (one 32-bit store each; the
    // eight swizzled row bases of the pair are formed once)
    const uint32_t ct = (warp < 4 ? warp - 2u : warp - 14u) * 32u + lane;
    bool ok = true;
    for (uint32_t j = 0;; j++) {
      if (!persist && j >= nloc) break;
      const uint32_t s = j % t.nslots;
      if (!warp_wait(&raw_full[s], (j / t.nslots) & 1u, sflag)) { ok = false; break; }
      if (persist && meta[s].gate == kNoGate) {   // release the issuer's wait on this slot, then stop
        __syncwarp();
        if (lane == 0) mbar_arrive(&img_full[s]);
        break;
      }
      const uint32_t* B = braw_of(s);
      uint8_t* img = img_of(s);
      for (uint32_t P = ct; P < Ng / 2; P += kSmConvThreads) {
        const uint32_t w = P >> 4, c = P & 15u;
        uint32_t x0[8], x1[8];
        ld_row(B + (32u * w + c) * W, W, x0);
        ld_row(B + (32u * w + c + 16u) * W, W, x1);
        const uint32_t f2 = b_factor(c);
        const uint32_t p0 = 2u * P, kin = p0 & 63u, chunk = kin >> 3;
        uint8_t* base = img + (p0 >> 6) * (t.ncols * 128u) + (kin & 7u) * 2u;
        uint8_t* rb[8];
#pragma unroll
        for (uint32_t r = 0; r < 8; r++) rb[r] = base + r * 128u + ((chunk ^ r) << 4);
#pragma unroll
        for (uint32_t e = 0; e < 8u / LL; e++) {
          if (e < NP1) {
#pragma unroll
            for (uint32_t wl = 0; wl < (uint32_t)LL; wl++) {
#pragma unroll
              for (uint32_t by = 0; by < 4; by++) {
                const uint32_t n = e * kDig + wl * 4u + by;
                const uint32_t sel = by | (by << 4) | ((4u + by) << 8) | ((4u + by) << 12);
                const uint32_t v =
                    (__byte_perm(x0[e * LL + wl], x1[e * LL + wl], sel) & 0x00FF00FFu) | 0x64006400u;
                *(uint32_t*)(rb[n & 7u] + (n >> 3) * 1024u) = hmul2(hsub2(v, 0x64006400u), f2);
              }
            }
          }
        }
      }
      fence_proxy_async_smem();   // generic-proxy writes -> the MMA's reads
      __syncwarp();
      if (lane == 0) mbar_arrive(&img_full[s]);
    }
    if (!ok && lane == 0) *sflag = 1;

  } else if (warp >= kSmExpWarp0 && warp < kSmEpiWarp0) {
    // ------------------------------------------------------------ A expanders
    const uint32_t q = warp & 3u;
    bool ok = true;
    uint32_t j = 0, m = 0, st = 0, stph = 0;
    for (uint32_t it = 0;; it++) {
      if (!persist && it >= items) break;
      const uint32_t s = j % t.nslots;
      if (m == 0) {
        if (!warp_wait(&raw_full[s], (j / t.nslots) & 1u, sflag)) { ok = false; break; }
        if (persist && meta[s].gate == kNoGate) break;
      }
      if (it >= t.nastages && !warp_wait(&afree[st], stph ^ 1u, sflag)) { ok = false; break; }
      tc_fence_after();
      const uint32_t r0 = m * 128u + q * 32u;
      if (r0 < Ng) {   // warp-uniform: Ng is a multiple of 32
        const uint32_t i = r0 + lane;
        uint32_t x[8];
        ld_row(araw_of(s) + i * W, W, x);
        if (meta[s].flags & 1u) {   // P - A, borrows inside each element
          const uint32_t pidx = (i / kEll) * LL + (i % kEll) / 32, pval = 1u << (i % 32);
          uint32_t borrow = 0;
#pragma unroll
          for (uint32_t w = 0; w < 8; w++) {
            if (w < W) {
              if (w % LL == 0) borrow = 0;
              const uint64_t dv = (uint64_t)(w == pidx ? pval : 0u) - x[w] - borrow;
              x[w] = (uint32_t)dv;
              borrow = (uint32_t)(dv >> 63);
            }
          }
        }
        const uint32_t col = tmem + ((q * 32u) << 16) + t.acc0 + st * t.acols;
#pragma unroll
        for (uint32_t w = 0; w < 8; w++) {
          if (w < W) {
            uint32_t v[16];
            bits_to_pairs(x[w], v);
            tmem_st_x16(col + 16u * w, v);
          }
        }
        tmem_wait_st();
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&afull[st]);
      if (++st == t.nastages) { st = 0; stph ^= 1u; }
      if (++m == t.mt) { m = 0; j++; }
    }
    if (!ok && lane == 0) *sflag = 1;

  } else if (warp >= kSmEpiWarp0 && warp < kSmEpiWarp0 + kSmEpiWarps) {
    // -------------------------------------------------------------- epilogue
    // warp (q, h): rows 32 q .. 32 q + 31 of each item, elements h, h + 2, ...
    const uint32_t q = warp & 3u, h = (warp - kSmEpiWarp0) >> 2;
    const bool storer = !persist && warp == kSmEpiWarp0 && lane == 0;
    const uint32_t tlane = tmem + ((q * 32u) << 16);
    // every accumulator slot starts at the bias (this warp's lanes and
    // elements); the arrival frees each slot for its first item
    for (uint32_t c = 0; c < t.nacc; c++) {
      for (uint32_t e = h; e < NP1; e += 2)
#pragma unroll
        for (uint32_t k = 0; k < (uint32_t)LL; k++) tmem_st_x4(tlane + c * t.ncols + e * kDig + 4u * k, kAccBiasBits);
    }
    tmem_wait_st();
    tc_fence_before();
    __syncwarp();
    if (lane == 0)
      for (uint32_t c = 0; c < t.nacc; c++) mbar_arrive(&accfree[c]);
    bool ok = true;
    uint32_t j = 0, m = 0, acc = 0, accph = 0;
    for (uint32_t it = 0;; it++) {
      if (!persist && it >= items) break;
      const uint32_t s = j % t.nslots;
      // the slot's metadata was published with raw_full (still this gate's phase)
      if (m == 0) {
        if (!warp_wait(&raw_full[s], (j / t.nslots) & 1u, sflag)) { ok = false; break; }
        if (persist && meta[s].gate == kNoGate) break;
      }
      if (!warp_wait(&accfull[acc], accph, sflag)) { ok = false; break; }
      tc_fence_after();
      const SlotMeta md = meta[s];
      const uint32_t r0 = m * 128u + q * 32u;
      const uint32_t taddr = tlane + acc * t.ncols;
      if (r0 < Ng) {
        const bool one = md.o0 != REF_NONE, two = md.o1 != REF_NONE;
        const uint32_t i = r0 + lane;
        uint32_t* Arow = araw_of(s) + i * W;
        uint32_t* Brow = braw_of(s) + i * W;
        // persistent form: outputs straight to their global rows (published
        // after a fence, no bulk-store completion to wait for); otherwise in
        // place over the slot's rows, leaving by bulk stores
        uint32_t* G0 = persist && one ? ct_ptr(a, md.o0) + (uint64_t)i * W : nullptr;
        uint32_t* G1 = persist && two ? ct_ptr(a, md.o1) + (uint64_t)i * W : nullptr;
        for (uint32_t e = h; e < NP1; e += 2) {
          uint32_t v[16];
          tmem_ld16(taddr + e * kDig, v);
          uint32_t av[LL], bv[LL], o0[LL], o1[LL];
          ld_elem<LL>(Arow + e * LL, av);
          ld_elem<LL>(Brow + e * LL, bv);
          // K words, unnormalised: S0 + S1 2^8 + S2 2^16 + S3 2^24 < 2^41
          uint64_t kw[LL];
#pragma unroll
          for (uint32_t wl = 0; wl < (uint32_t)LL; wl++) {
            const uint32_t lo01 = v[4 * wl] + (v[4 * wl + 1] << 8), lo23 = v[4 * wl + 2] + (v[4 * wl + 3] << 8);
            kw[wl] = (uint64_t)lo01 + ((uint64_t)lo23 << 16) - kWordBias;
          }
          if (md.kind == kKindHA) {   // XOR = A + B - 2K, AND = K
            int64_t cx = 0;
            uint64_t ca = 0;
#pragma unroll
            for (uint32_t wl = 0; wl < (uint32_t)LL; wl++) {
              const int64_t tx = (int64_t)av[wl] + (int64_t)bv[wl] - 2 * (int64_t)kw[wl] + cx;
              o0[wl] = (uint32_t)tx;
              cx = tx >> 32;
              const uint64_t ta = kw[wl] + ca;
              o1[wl] = (uint32_t)ta;
              ca = ta >> 32;
            }
          } else if (md.kind == kKindOR) {   // A + B - K
            int64_t co = 0;
#pragma unroll
            for (uint32_t wl = 0; wl < (uint32_t)LL; wl++) {
              const int64_t to = (int64_t)av[wl] + (int64_t)bv[wl] - (int64_t)kw[wl] + co;
              o0[wl] = (uint32_t)to;
              co = to >> 32;
            }
          } else {
            const uint32_t code = md.code;
            const int c00 = nib(code, 0), c01 = nib(code, 1), c02 = nib(code, 2), c03 = nib(code, 3);
            const int c10 = nib(code, 4), c11 = nib(code, 5), c12 = nib(code, 6), c13 = nib(code, 7);
            // a term c x (c small, x < 2^32) is c (x - 2^31) + c 2^31: one signed
            // 32 x 32 -> 64 multiply-add, the constants summed once per output
            const int64_t bias0 = (int64_t)(c01 + c02 + c03) << 31, bias1 = (int64_t)(c11 + c12 + c13) << 31;
            const uint32_t pe = i / kEll, pw = (i % kEll) / 32;
            const int64_t pv = (int64_t)1 << (i % 32);
            int32_t carry0 = 0, carry1 = 0;
#pragma unroll
            for (uint32_t wl = 0; wl < (uint32_t)LL; wl++) {
              const int32_t khi = (int32_t)(kw[wl] >> 32);
              const int32_t xa = (int32_t)(av[wl] ^ 0x80000000u), xb = (int32_t)(bv[wl] ^ 0x80000000u);
              const int32_t xk = (int32_t)((uint32_t)kw[wl] ^ 0x80000000u);
              const bool pat = e == pe && wl == pw;
              int64_t t0 = bias0 + carry0;
              t0 += (int64_t)c01 * xa;
              t0 += (int64_t)c02 * xb;
              t0 += (int64_t)c03 * xk;
              if (pat) t0 += c00 * pv;
              carry0 = (int32_t)(t0 >> 32) + c03 * khi;
              o0[wl] = (uint32_t)t0;
              int64_t t1 = bias1 + carry1;
              t1 += (int64_t)c11 * xa;
              t1 += (int64_t)c12 * xb;
              t1 += (int64_t)c13 * xk;
              if (pat) t1 += c10 * pv;
              carry1 = (int32_t)(t1 >> 32) + c13 * khi;
              o1[wl] = (uint32_t)t1;
            }
          }
          if (persist) {
            if (one) st_elem_global<LL>(G0 + e * LL, o0);   // output 0
            if (two) st_elem_global<LL>(G1 + e * LL, o1);   // output 1
          } else {
            if (one) st_elem<LL>(Arow + e * LL, o0);
            if (two) st_elem<LL>(Brow + e * LL, o1);
          }
        }
      }
      // the slot's next item starts again from the bias (every warp, its own
      // lanes and elements, whether or not its rows were live)
      for (uint32_t e = h; e < NP1; e += 2)
#pragma unroll
        for (uint32_t k = 0; k < (uint32_t)LL; k++) tmem_st_x4(taddr + e * kDig + 4u * k, kAccBiasBits);
      tmem_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&accfree[acc]);
      if (++acc == t.nacc) { acc = 0; accph ^= 1u; }
      if (++m == t.mt) {
        // the gate is complete; the arrival orders this warp's output stores
        // before the publisher's gpu-scope fence (persistent form), or the
        // in-place outputs before the bulk stores read them
        if (!persist) fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&epi_done[s]);
        bool bad = false;
        if (storer) {
          if (mbar_wait_flag(&epi_done[s], (j / t.nslots) & 1u, sflag)) {
            if (md.o0 != REF_NONE) bulk_s2g(ct_ptr(a, md.o0), araw_of(s), t.raw_bytes);
            if (md.o1 != REF_NONE) bulk_s2g(ct_ptr(a, md.o1), braw_of(s), t.raw_bytes);
            bulk_commit();
            bulk_wait_read();
            mbar_arrive(&slot_free[s]);
          } else {
            bad = true;
          }
        }
        if (!persist && __any_sync(0xFFFFFFFFu, bad)) { ok = false; break; }   // the whole warp leaves together
        m = 0;
        j++;
      }
    }
    if (storer) bulk_wait_all();
    if (!ok && lane == 0) *sflag = 1;

  } else if (persist && warp == kSmPubWarp) {
    // -------------------------------------------------------------- publisher
    // gates in ring order (lane 0 works, the warp keeps step)
    bool ok = true;
    const uint32_t ep = persist ? *a.epoch : 0u;
    for (uint32_t j = 0;; j++) {
      const uint32_t s = j % t.nslots, ph = (j / t.nslots) & 1u;
      if (!warp_wait(&raw_full[s], ph, sflag)) { ok = false; break; }
      if (meta[s].gate == kNoGate) break;
      if (!warp_wait(&epi_done[s], ph, sflag)) { ok = false; break; }
      if (lane == 0) {
        const uint32_t gate = meta[s].gate;
        const uint32_t lev = a.glev[gate];
        // every epilogue warp's output stores happen before its arrival on
        // epi_done, observed above; one gpu-scope fence makes both writes
        // below release patterns (flag for the gate's readers, count for the
        // level window)
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(a.gflag + gate), "r"(ep) : "memory");
        asm volatile("red.relaxed.gpu.global.add.u64 [%0], 1;" ::"l"(a.ldone + lev) : "memory");
        mbar_arrive(&slot_free[s]);
      }
      __syncwarp();
    }
    if (!ok && lane == 0) *sflag = 1;
  }

  __syncthreads();
  if (*sflag) {
    if (tid == 0 && a.err) atomicExch(a.err, KERR_MMA_TIMEOUT);
    if (warp == 0) mbar_wait_bounded(drain, 0);   // own MMAs drain before TMEM is freed
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, kSmTmemCols);
  }
}

}  // namespace sfft

namespace sfft {

namespace {

// Ring slots used when no tuned value is set (sfft_autotune stores one per
// shape).
constexpr uint32_t kSmDefaultSlots = 4;

uint32_t sm_smem_bytes(uint32_t slot_bytes, uint32_t nslots) {
  return 1024u + nslots * slot_bytes + kSmMaxSlots * 32u + kSmBars * 8u;   // + slot metadata
}

// nslots 0: the tuned or default ring depth.
bool make_sm_shape(const KArgs& a, uint32_t nslots, SmShape* t) {
  // Ng 64 or 96: one 128-row item whose upper lane quarters carry no rows
  // (their expanders and epilogue warps skip the work, not the barriers)
  if (a.Ng < 64 || a.Ng > 256 || a.L == 0 || a.L > 4 || a.ell != 32 * a.L || a.W % a.L) return false;
  const uint32_t NP1 = a.W / a.L;
  if (NP1 < 2 || a.W > 8) return false;
  t->mt = (a.Ng + 127) / 128;
  t->ksteps = a.Ng / 16;
  t->atoms = (a.Ng + 63) / 64;
  t->dig = a.ell / 8;
  t->ncols = (NP1 * t->dig + 15) / 16 * 16;
  if (t->ncols > 256) return false;
  t->img_bytes = t->atoms * t->ncols * 128u;
  t->raw_bytes = a.Ng * a.W * 4u;
  t->slot_bytes = (t->img_bytes + 2u * t->raw_bytes + 1023u) / 1024u * 1024u;
  t->acols = a.Ng / 2;
  t->nastages = std::min<uint32_t>(kSmMaxAStages, (kSmTmemCols - 2u * t->ncols) / t->acols);
  if (t->nastages < 2) return false;
  t->nacc = std::min<uint32_t>(kSmMaxAcc, (kSmTmemCols - t->nastages * t->acols) / t->ncols);
  if (t->nacc < 2) return false;
  t->acc0 = t->nacc * t->ncols;
  uint32_t ns = nslots ? nslots : kSmDefaultSlots;
  while (ns > 1 && sm_smem_bytes(t->slot_bytes, ns) > kSmMaxSmem) ns--;
  if (ns < 2 || ns > kSmMaxSlots) return false;
  t->nslots = ns;
  // at least half the opt-in: one CTA per SM (each allocates all 512
  // tensor-memory columns)
  t->smem_bytes = std::max(sm_smem_bytes(t->slot_bytes, ns), kSmMaxSmem / 2 + 1024u);
  return true;
}

// Per device: SM count and whether the kernels' shared-memory opt-in is set.
struct SmDevice {
  int sms = 0;
  bool configured = false;
};
std::mutex g_sm_mu;
SmDevice g_sm_dev[64];
uint32_t g_sm_tuned_slots[64][4] = {};   // [device][limbs - 1], 0 = untuned

int sm_device(SmDevice** out, int* ordinal) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return fail(SFFT_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_sm_mu);
  SmDevice& d = g_sm_dev[dev];
  if (!d.configured) {
    e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
    const void* fns[] = {(const void*)k_gate_sm<1, false>, (const void*)k_gate_sm<2, false>,
                         (const void*)k_gate_sm<3, false>, (const void*)k_gate_sm<4, false>,
                         (const void*)k_gate_sm<1, true>,  (const void*)k_gate_sm<2, true>,
                         (const void*)k_gate_sm<3, true>,  (const void*)k_gate_sm<4, true>};
    for (const void* fn : fns)
      if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmMaxSmem);
    if (e != cudaSuccess) return cuda_fail(e, "small-ciphertext kernel attributes");
    d.configured = true;
  }
  *out = &d;
  if (ordinal) *ordinal = dev;
  return SFFT_OK;
}

}  // namespace

bool sm_supported(const KArgs& a) {
  SmShape t;
  return make_sm_shape(a, 0, &t);
}

uint32_t sm_digit_columns(const KArgs& a) {
  SmShape t;
  if (!make_sm_shape(a, 0, &t)) return 0;
  return (a.W / a.L) * t.dig;
}

int launch_gates_sm_slots(const KArgs& a, uint32_t nslots, cudaStream_t st) {
  if (a.n == 0) return SFFT_OK;
  SmDevice* dev = nullptr;
  int ordinal = 0;
  int rc = sm_device(&dev, &ordinal);
  if (rc) return rc;
  if (!nslots) {
    std::lock_guard<std::mutex> lk(g_sm_mu);
    nslots = g_sm_tuned_slots[ordinal][(a.L - 1) & 3];
  }
  SmShape t{};
  if (!make_sm_shape(a, nslots, &t))
    return fail(SFFT_EPARAM, "small-ciphertext kernel does not support this shape");
  const uint64_t blocks = std::min<uint64_t>(a.n, (uint64_t)dev->sms);
  Timer* tm = static_cast<Timer*>(a.timer);
  if (tm) cudaEventRecord(tm->next(kTimeGate), st);
  if (a.glev) {   // one launch across levels
    switch (a.L) {
      case 1: k_gate_sm<1, true><<<(unsigned)blocks, kSmThreadsPersist, t.smem_bytes, st>>>(a, t); break;
      case 2: k_gate_sm<2, true><<<(unsigned)blocks, kSmThreadsPersist, t.smem_bytes, st>>>(a, t); break;
      case 3: k_gate_sm<3, true><<<(unsigned)blocks, kSmThreadsPersist, t.smem_bytes, st>>>(a, t); break;
      default: k_gate_sm<4, true><<<(unsigned)blocks, kSmThreadsPersist, t.smem_bytes, st>>>(a, t); break;
    }
  } else {
    switch (a.L) {
      case 1: k_gate_sm<1, false><<<(unsigned)blocks, kSmThreads, t.smem_bytes, st>>>(a, t); break;
      case 2: k_gate_sm<2, false><<<(unsigned)blocks, kSmThreads, t.smem_bytes, st>>>(a, t); break;
      case 3: k_gate_sm<3, false><<<(unsigned)blocks, kSmThreads, t.smem_bytes, st>>>(a, t); break;
      default: k_gate_sm<4, false><<<(unsigned)blocks, kSmThreads, t.smem_bytes, st>>>(a, t); break;
    }
  }
  if (tm) cudaEventRecord(tm->next(kTimeGate), st);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SFFT_OK : cuda_fail(e, "small-ciphertext gate kernel launch");
}

int launch_gates_sm(const KArgs& a, cudaStream_t st) { return launch_gates_sm_slots(a, 0, st); }

// Ring depth used from now on for this device and limb count (0 = default).
int sm_set_tuned_slots(uint32_t L, uint32_t nslots) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64 || L == 0 || L > 4) return fail(SFFT_EINVAL, "bad device or limb count");
  std::lock_guard<std::mutex> lk(g_sm_mu);
  g_sm_tuned_slots[dev][L - 1] = nslots;
  return SFFT_OK;
}

}  // namespace sfft

// ---------------------------------------------------------------------------
// Autotuner: ring depth (gates in flight per CTA) of the small-ciphertext
// kernel, timed on one level of random products.
// ---------------------------------------------------------------------------
namespace sfft {

namespace {

__global__ void k_fill_random(uint32_t* p, uint64_t n, uint64_t seed) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;   // SplitMix64 finaliser
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    p[i] = (uint32_t)(z ^ (z >> 31));
  }
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { cudaFree(p); }
};

}  // namespace

}  // namespace sfft

using namespace sfft;

extern "C" int sfft_small_kernel_set_slots(uint32_t ell, uint32_t nslots) {
  if (nslots == 1 || nslots > kSmMaxSlots) return fail(SFFT_EINVAL, "ring depth must be 0 or 2..8");
  if (ell == 0 || ell % 32 || ell > 128) return fail(SFFT_EINVAL, "ell must be 32, 64, 96 or 128");
  return sm_set_tuned_slots(ell / 32, nslots);
}

extern "C" int sfft_autotune_small(const sfft_params* p, uint64_t n_gates, uint32_t reps,
                                   uint32_t* best_slots, double* h_us_per_gate) {
  Shape s;
  int rc = make_shape(p, &s, false);
  if (rc) return rc;
  KArgs a = make_args(s);
  SmShape t;
  if (!make_sm_shape(a, 0, &t)) return fail(SFFT_EPARAM, "the small-ciphertext kernel does not take these parameters");
  if (n_gates == 0 || n_gates > (1u << 24)) return fail(SFFT_EINVAL, "n_gates must be 1 .. 2^24");
  if (reps == 0) reps = 3;
  const uint64_t words = n_gates * s.ctw;
  DevBuf ab, bb, o0, o1, dd, da, de;
  std::vector<GateDesc> desc(n_gates);
  std::vector<GateAux> aux(n_gates);
  for (uint64_t g = 0; g < n_gates; g++) {   // half adders, every other A complemented
    desc[g] = GateDesc{make_ref(REG_SCRATCH, (uint32_t)g), make_ref(REG_IN, (uint32_t)g),
                       make_ref(REG_OUT, (uint32_t)g), make_ref(REG_GEN, (uint32_t)g)};
    aux[g].code = (uint32_t)pack_code(0, 1, 1, -2) | ((uint32_t)pack_code(0, 0, 0, 1) << 16);
    aux[g].flags = g & 1u;
  }
  cudaError_t e = cudaMalloc(&ab.p, words * 4);
  if (e == cudaSuccess) e = cudaMalloc(&bb.p, words * 4);
  if (e == cudaSuccess) e = cudaMalloc(&o0.p, words * 4);
  if (e == cudaSuccess) e = cudaMalloc(&o1.p, words * 4);
  if (e == cudaSuccess) e = cudaMalloc(&de.p, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(de.p, 0, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(e, "autotune buffers");
  if ((rc = upload(desc.data(), desc.size() * sizeof(GateDesc), &dd.p))) return rc;
  if ((rc = upload(aux.data(), aux.size() * sizeof(GateAux), &da.p))) return rc;
  k_fill_random<<<1024, 256>>>((uint32_t*)ab.p, words, 1);
  k_fill_random<<<1024, 256>>>((uint32_t*)bb.p, words, 2);
  a.desc = (const GateDesc*)dd.p;
  a.aux = (const GateAux*)da.p;
  a.n = n_gates;
  a.base[REG_SCRATCH] = (uint32_t*)ab.p;
  a.base[REG_IN] = (uint32_t*)bb.p;
  a.base[REG_OUT] = (uint32_t*)o0.p;
  a.base[REG_GEN] = (uint32_t*)o1.p;
  a.err = (int*)de.p;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 0;
  uint32_t best_ns = 0;
  for (uint32_t ns = 2; ns <= kSmMaxSlots; ns++) {
    if (h_us_per_gate) h_us_per_gate[ns - 1] = 0;
    SmShape c;
    if (!make_sm_shape(a, ns, &c) || c.nslots != ns) continue;
    if ((rc = launch_gates_sm_slots(a, ns, 0))) break;   // warm-up
    double ms_min = 1e30;
    for (uint32_t r = 0; r < reps && !rc; r++) {
      cudaEventRecord(e0, 0);
      rc = launch_gates_sm_slots(a, ns, 0);
      cudaEventRecord(e1, 0);
      cudaEventSynchronize(e1);
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      ms_min = std::min<double>(ms_min, ms);
    }
    if (rc) break;
    const double us = ms_min * 1000.0 / (double)n_gates;
    if (h_us_per_gate) h_us_per_gate[ns - 1] = us;
    if (!best_ns || us < best) {
      best = us;
      best_ns = ns;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  e = cudaDeviceSynchronize();
  if (!rc && e != cudaSuccess) rc = cuda_fail(e, "autotune");
  if (!rc) rc = check_device_error(a.err, 0);
  if (rc) return rc;
  if (best_slots) *best_slots = best_ns;
  return sm_set_tuned_slots(s.L, best_ns);
}
