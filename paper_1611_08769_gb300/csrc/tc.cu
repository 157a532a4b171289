// Gate product on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// The GSW product K = BitDecomp(A~) B' (Sec. 7: an N x N matrix product per
// gate) is a dense contraction of a {0,1} matrix with B''s digits. Splitting
// every 32-bit limb of B' into its four bytes gives, per output row i and
// byte column n (byte n%4 of word n/4),
//     S[i][n] = sum_k bit_k(A~_i) * byte_n(B'_k)  <  255 Ng  < 2^24,
// so an fp16 x fp16 -> fp32 MMA computes it exactly. Operands are encoded
// without subnormals: a bit as fp16 1.0, a byte b as fp16 (1024 + b) (bit
// pattern 0x6400 | b); the 1024 * popcount(A~_i) term is removed in the
// epilogue. The epilogue forms K[i][w] = sum_b S[i][4w+b] 2^(8b) and adds the
// linear terms c0 P + c1 A + c2 B with the limb carries of each element,
// exactly as the integer kernel does.
//
// One CTA (8 warps) computes a 128-row tile of one gate's output over all
// byte columns:
//  * the A~ tile (128 rows, contiguous in global memory) arrives by one bulk
//    copy (cp.async.bulk + mbarrier transaction count) and is complemented in
//    place when the descriptor asks for P - A;
//  * B' is consumed in 64-row slices (contiguous); slices are bulk-copied
//    into a 3-deep shared-memory ring ahead of use;
//  * per slice, the threads expand A bits and B bytes into 128B-swizzled
//    K-major fp16 tiles (two buffers) and one thread issues the tcgen05.mma
//    chain into the TMEM accumulator and commits to an mbarrier; the next
//    slice is expanded while the tensor core runs;
//  * the epilogue reads the accumulator with tcgen05.ld, takes A~ and the
//    tile's B' rows (bulk-copied) from shared memory, builds the two output
//    tiles in shared memory and writes each back with one bulk store.
// Every mbarrier wait is bounded (~2 s); on timeout the kernel records
// KERR_MMA_TIMEOUT, waits (bounded) for its own MMAs, frees its TMEM and
// returns.
#include <cuda_runtime.h>

#include <cstdint>

#include "common.h"
#include "kargs.h"
#include "plan.h"
#include "rng.h"

namespace sfft {

namespace {

constexpr int kThreads = 256;
constexpr int kTileM = 128;
constexpr int kBK = 64;                        // K elements per slice (128 bytes of fp16)
constexpr uint32_t kSpinLimit = 1u << 26;
constexpr uint64_t kWaitNs = 2000000000ull;    // bound of any single mbarrier wait
constexpr uint32_t kMaxSmem = 232448;          // 227 KB opt-in per CTA

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits for the phase with the given parity, giving up after ~2 s (or an
// iteration cap, whichever comes first).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0; it < kSpinLimit; it++) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 255u && global_ns() - t0 > kWaitNs) return false;
  }
  return false;
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Bulk copy global -> shared, completing `bytes` transactions on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Bulk copy shared -> global (bulk-group completion).
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
               "r"(smem_u32(src)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, fp16 inputs, fp32 accumulate.
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15},"
      " [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (tile base 1024-byte aligned).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                    // leading byte offset (unused when swizzled)
  d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset
  d |= (uint64_t)1 << 46;                    // descriptor version
  d |= (uint64_t)2 << 61;                    // SWIZZLE_128B
  return d;
}

// Instruction descriptor of kind::f16: F16 x F16 -> F32, both K-major.
__host__ __device__ constexpr uint32_t idesc_f16(uint32_t M, uint32_t N) {
  return (1u << 4) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

// Byte offset of 16-byte chunk `c` (K elements 8c .. 8c+7) of row `r` in a
// 128B-swizzled K-major tile.
__device__ __forceinline__ uint32_t sw128_off(uint32_t r, uint32_t c) {
  return r * 128u + ((c ^ (r & 7u)) << 4);
}

__device__ __forceinline__ uint32_t p_word(uint32_t i, uint32_t j, uint32_t l, uint32_t ell) {
  return (j == i / ell && l == (i % ell) / 32) ? (1u << (i % 32)) : 0u;
}

__device__ __forceinline__ int nib(uint32_t code, int k) {
  return (int)((int32_t)(code << (28 - 4 * k)) >> 28);
}

// Two fp16 1.0/0.0 values from two bits: bit0 -> low half, bit1 -> high half.
__device__ __forceinline__ uint32_t bits2h(uint32_t x) {
  return ((x & 1u) * 0x3C00u) | (((x >> 1) & 1u) * 0x3C000000u);
}

}  // namespace

struct TcShape {
  uint32_t nd, ndpad, tmem_cols, mtiles, kblocks, nstages;
  uint32_t n0_len, n1_len;   // MMA N of the two column chunks (n1_len 0 if one chunk)
  uint32_t stage_bytes, ring_bytes, smem_bytes;
};

namespace {

// Shared-memory layout for W words per row and ring depth ns.
__host__ __device__ inline void tc_layout(uint32_t W, uint32_t ndpad, uint32_t ns, uint32_t* stage,
                                          uint32_t* ring, uint32_t* total) {
  *stage = 16384u + ndpad * 128u;                      // expanded A tile + expanded B tile
  *ring = (uint32_t)kBK * W * 4u;                      // one raw 64-row slice of B'
  const uint32_t tileA = (uint32_t)kTileM * W * 4u;
  uint32_t ring_total = ns * *ring;
  if (ring_total < tileA) ring_total = tileA;          // the ring also holds the epilogue's B rows
  *total = 1024u + 2u * *stage + ring_total + tileA + kTileM * 4u + 128u;
}

}  // namespace

__global__ void __launch_bounds__(kThreads, 1) k_gate_tc(KArgs a, TcShape t) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t W = a.W, L = a.L, NP1 = W / L;
  uint8_t* stage0 = smem;
  uint8_t* ring = smem + 2 * t.stage_bytes;
  uint32_t ring_total = t.nstages * t.ring_bytes;
  if (ring_total < (uint32_t)kTileM * W * 4u) ring_total = kTileM * W * 4u;
  uint32_t* tileA = (uint32_t*)(ring + ring_total);                // A~ rows of the tile
  uint32_t* spop = tileA + kTileM * W;                              // popcount per row
  uint64_t* bars = (uint64_t*)(spop + kTileM);
  uint64_t* full = bars;                                            // [nstages] ring slots
  uint64_t* mmab = bars + 4;                                        // [2] MMA commits
  uint64_t* abar = bars + 6;                                        // A tile arrived
  uint64_t* ebar = bars + 7;                                        // epilogue B rows arrived
  uint32_t* tslot = (uint32_t*)(bars + 8);

  const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint64_t g = blockIdx.x / t.mtiles;
  const uint32_t row0 = (blockIdx.x % t.mtiles) * kTileM;
  if (g >= a.n) return;
  const uint32_t rows = (a.Ng - row0) < (uint32_t)kTileM ? (a.Ng - row0) : (uint32_t)kTileM;
  const GateDesc d = a.desc[g];
  const GateAux x = a.aux[g];
  const bool gen = (d.a >> 30) == REG_GEN;
  const uint32_t* A = gen ? nullptr : a.base[d.a >> 30] + (uint64_t)(d.a & SLOT_MASK) * a.ctw;
  const uint64_t gst = gen ? stream_out(a.gen_state, d.a & SLOT_MASK) : 0;
  const uint32_t* B = a.base[d.b >> 30] + (uint64_t)(d.b & SLOT_MASK) * a.ctw;
  const bool comp = (x.flags & 1u) != 0;

  if (tid == 0) {
    for (int b = 0; b < 8; b++) mbar_init(&bars[b], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(tslot, t.tmem_cols);
  __syncthreads();
  if (tid == 0) {
    if (!gen) {
      mbar_expect_tx(abar, rows * W * 4u);
      bulk_g2s(tileA, A + (uint64_t)row0 * W, rows * W * 4u, abar);
    }
    for (uint32_t s = 0; s < t.nstages && s < t.kblocks; s++) {
      const uint32_t krows = (a.Ng - s * kBK) < (uint32_t)kBK ? (a.Ng - s * kBK) : (uint32_t)kBK;
      mbar_expect_tx(&full[s], krows * W * 4u);
      bulk_g2s(ring + s * t.ring_bytes, B + (uint64_t)s * kBK * W, krows * W * 4u, &full[s]);
    }
  }
  // zero the padded byte-column rows of both expanded B tiles (never rewritten)
  for (uint32_t e = tid; e < (t.ndpad - t.nd) * 32u; e += kThreads) {
    const uint32_t r = t.nd + e / 32, c = e % 32;
    ((uint32_t*)(stage0 + 16384u + r * 128u))[c] = 0;
    ((uint32_t*)(stage0 + t.stage_bytes + 16384u + r * 128u))[c] = 0;
  }
  bool timed_out = false;
  if (gen) {
    for (uint32_t e = tid; e < kTileM * W; e += kThreads) {
      const uint32_t r = e / W, w = e % W;
      tileA[e] = r < rows ? r_word(gst, (uint64_t)(row0 + r) * W + w) : 0u;
    }
  } else {
    timed_out = !mbar_wait_bounded(abar, 0);
    for (uint32_t e = rows * W + tid; e < kTileM * W; e += kThreads) tileA[e] = 0;
  }
  __syncthreads();
  // Complement (P - A) row by row with the borrow chain of each element; popcount.
  if (tid < kTileM) {
    const uint32_t r = tid, i = row0 + r;
    uint32_t pc = 0, borrow = 0;
    for (uint32_t w = 0; w < W; w++) {
      uint32_t v = tileA[r * W + w];
      if (comp && r < rows) {
        const uint32_t l = w % L;
        if (l == 0) borrow = 0;
        const uint64_t dv = (uint64_t)p_word(i, w / L, l, a.ell) - v - borrow;
        v = (uint32_t)dv;
        borrow = (uint32_t)(dv >> 63);
        tileA[r * W + w] = v;
      }
      pc += __popc(v);
    }
    spop[r] = pc;
  }
  tc_fence_before();
  bool ok = !__syncthreads_or(timed_out);
  tc_fence_after();
  const uint32_t tmem = *tslot;

  const uint32_t idesc0 = idesc_f16(kTileM, t.n0_len), idesc1 = idesc_f16(kTileM, t.n1_len);
  for (uint32_t kb = 0; ok && kb < t.kblocks; kb++) {
    const uint32_t s = kb & 1, slot = kb % t.nstages;
    uint8_t* sA = stage0 + s * t.stage_bytes;
    uint8_t* sB = sA + 16384u;
    const uint32_t* raw = (const uint32_t*)(ring + slot * t.ring_bytes);
    // the MMAs of slice kb-2 read this stage; slice kb's raw rows must have landed
    bool w_ok = kb < 2 || mbar_wait_bounded(&mmab[s], ((kb - 2) >> 1) & 1);
    w_ok = w_ok && mbar_wait_bounded(&full[slot], (kb / t.nstages) & 1);
    const uint32_t krows = (a.Ng - kb * kBK) < (uint32_t)kBK ? (a.Ng - kb * kBK) : (uint32_t)kBK;
    // A~ slice: 128 rows x 64 bits -> fp16 {0,1}; task = (row, 16-byte chunk)
    for (uint32_t e = tid; e < kTileM * 8u; e += kThreads) {
      const uint32_t r = e >> 3, c = e & 7;
      const uint32_t kbit = kb * kBK + c * 8;
      const uint32_t wi = kbit >> 5;
      const uint32_t byte = wi < W ? (tileA[r * W + wi] >> (kbit & 31)) & 0xFFu : 0u;
      uint4 v;
      v.x = bits2h(byte);
      v.y = bits2h(byte >> 2);
      v.z = bits2h(byte >> 4);
      v.w = bits2h(byte >> 6);
      *(uint4*)(sA + sw128_off(r, c)) = v;
    }
    // B slice: raw rows k (64) -> byte columns n = 4w + b as fp16 (1024 + byte)
    for (uint32_t e = tid; e < 8u * W; e += kThreads) {
      const uint32_t c = e & 7, w = e >> 3;
      uint32_t xw[8];
#pragma unroll
      for (int q = 0; q < 8; q++) {
        const uint32_t k = c * 8 + q;
        xw[q] = k < krows ? raw[k * W + w] : 0u;
      }
#pragma unroll
      for (int b = 0; b < 4; b++) {
        // prmt: result byte 0 = byte b of the first word, byte 2 = byte b of the
        // second; mask to those bytes and add the 0x6400 (fp16 1024) magic.
        const uint32_t sel = (uint32_t)b | ((uint32_t)(b + 4) << 8);
        uint4 v;
        v.x = (__byte_perm(xw[0], xw[1], sel) & 0x00FF00FFu) | 0x64006400u;
        v.y = (__byte_perm(xw[2], xw[3], sel) & 0x00FF00FFu) | 0x64006400u;
        v.z = (__byte_perm(xw[4], xw[5], sel) & 0x00FF00FFu) | 0x64006400u;
        v.w = (__byte_perm(xw[6], xw[7], sel) & 0x00FF00FFu) | 0x64006400u;
        *(uint4*)(sB + sw128_off(4 * w + b, c)) = v;
      }
    }
    fence_proxy_async_smem();
    if (__syncthreads_or(!w_ok)) {
      ok = false;
      break;
    }
    if (tid == 0) {
      // refill the ring slot just consumed
      const uint32_t nk = kb + t.nstages;
      if (nk < t.kblocks) {
        const uint32_t nrows = (a.Ng - nk * kBK) < (uint32_t)kBK ? (a.Ng - nk * kBK) : (uint32_t)kBK;
        mbar_expect_tx(&full[slot], nrows * W * 4u);
        bulk_g2s(ring + slot * t.ring_bytes, B + (uint64_t)nk * kBK * W, nrows * W * 4u, &full[slot]);
      }
      tc_fence_after();
      const uint32_t a_base = smem_u32(sA), b_base = smem_u32(sB);
#pragma unroll
      for (uint32_t ks = 0; ks < kBK / 16; ks++) {
        const uint64_t ad = sw128_desc(a_base + ks * 32);
        mma_f16(tmem, ad, sw128_desc(b_base + ks * 32), idesc0, (kb | ks) != 0);
        if (t.n1_len)
          mma_f16(tmem + t.n0_len, ad, sw128_desc(b_base + t.n0_len * 128u + ks * 32), idesc1,
                  (kb | ks) != 0);
      }
      mma_commit(&mmab[s]);
    }
  }
  // B rows of this tile (linear term c2 B) into the ring, which is free now
  if (ok && tid == 0) {
    mbar_expect_tx(ebar, rows * W * 4u);
    bulk_g2s(ring, B + (uint64_t)row0 * W, rows * W * 4u, ebar);
  }
  const uint32_t last = t.kblocks - 1;
  if (ok) {
    bool w_ok = mbar_wait_bounded(&mmab[last & 1], (last >> 1) & 1);
    w_ok = w_ok && mbar_wait_bounded(ebar, 0);
    ok = !__syncthreads_or(!w_ok);
  }
  if (!ok) {
    if (tid == 0 && a.err) atomicExch(a.err, KERR_MMA_TIMEOUT);
    mbar_wait_bounded(&mmab[last & 1], (last >> 1) & 1);   // bounded: let own MMAs drain
  }
  tc_fence_after();

  if (ok) {
    // Epilogue: warp w reads TMEM lanes 32 (w % 4) ..; warps 0-3 and 4-7 take
    // alternate elements of the row. Outputs go to row-major tiles in the
    // (now idle) expanded stages.
    const uint32_t r = (warp & 3) * 32 + lane, i = row0 + r;
    const bool live = r < rows;
    const int64_t bias = 1024 * (int64_t)spop[r];
    const uint32_t* Bt = (const uint32_t*)ring;
    uint32_t* T0 = (uint32_t*)stage0;
    uint32_t* T1 = (uint32_t*)(stage0 + t.stage_bytes);
    uint32_t code0 = x.code & 0xFFFFu, code1 = x.code >> 16;
    int c00 = nib(code0, 0), c01 = nib(code0, 1), c02 = nib(code0, 2), c03 = nib(code0, 3);
    int c10 = nib(code1, 0), c11 = nib(code1, 1), c12 = nib(code1, 2), c13 = nib(code1, 3);
    if (comp) {  // the stored A is P - A~: c1 A = c1 P - c1 A~
      c00 += c01;
      c01 = -c01;
      c10 += c11;
      c11 = -c11;
    }
    const bool has0 = d.o0 != REF_NONE, has1 = d.o1 != REF_NONE;
    for (uint32_t j = warp >> 2; j < NP1; j += 2) {
      int64_t carry0 = 0, carry1 = 0;
      const uint32_t wbeg = j * L, wend = wbeg + L;
      for (uint32_t n0 = (4 * wbeg) & ~15u; n0 < 4 * wend; n0 += 16) {
        uint32_t v[16];
        tmem_ld16(tmem + (((warp & 3) * 32u) << 16) + n0, v);
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const uint32_t w = n0 / 4 + q;
          if (w < wbeg || w >= wend || !live) continue;
          int64_t k = 0;
#pragma unroll
          for (int b = 0; b < 4; b++) {
            const int64_t sv = (int64_t)__float2int_rn(__uint_as_float(v[4 * q + b])) - bias;
            k += sv << (8 * b);
          }
          const int64_t aw = (int64_t)tileA[r * W + w];
          const int64_t bw = (int64_t)Bt[r * W + w];
          const int64_t pw = (int64_t)p_word(i, j, w - wbeg, a.ell);
          if (has0) {
            const int64_t o = c03 * k + c01 * aw + c02 * bw + c00 * pw + carry0;
            T0[r * W + w] = (uint32_t)o;
            carry0 = o >> 32;
          }
          if (has1) {
            const int64_t o = c13 * k + c11 * aw + c12 * bw + c10 * pw + carry1;
            T1[r * W + w] = (uint32_t)o;
            carry1 = o >> 32;
          }
        }
      }
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      if (has0)
        bulk_s2g(a.base[d.o0 >> 30] + (uint64_t)(d.o0 & SLOT_MASK) * a.ctw + (uint64_t)row0 * W, T0,
                 rows * W * 4u);
      if (has1)
        bulk_s2g(a.base[d.o1 >> 30] + (uint64_t)(d.o1 & SLOT_MASK) * a.ctw + (uint64_t)row0 * W, T1,
                 rows * W * 4u);
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, t.tmem_cols);
  }
}

namespace {

bool make_tc_shape(const KArgs& a, TcShape* t) {
  if (a.Ng < 128) return false;
  t->nd = a.W * 4;
  t->ndpad = (t->nd + 15) / 16 * 16;
  if (t->ndpad > 512) return false;
  t->n0_len = t->ndpad < 256 ? t->ndpad : 256;
  t->n1_len = t->ndpad - t->n0_len;
  t->tmem_cols = 32;
  while (t->tmem_cols < t->ndpad) t->tmem_cols *= 2;
  t->mtiles = (a.Ng + kTileM - 1) / kTileM;
  t->kblocks = (a.Ng + kBK - 1) / kBK;
  for (uint32_t ns = 3; ns >= 2; ns--) {
    tc_layout(a.W, t->ndpad, ns, &t->stage_bytes, &t->ring_bytes, &t->smem_bytes);
    if (t->smem_bytes <= kMaxSmem) {
      t->nstages = ns;
      return true;
    }
  }
  return false;
}

}  // namespace

bool tc_supported(const KArgs& a) {
  TcShape t;
  return make_tc_shape(a, &t);
}

int launch_gates_tc(const KArgs& a, cudaStream_t st) {
  if (a.n == 0) return SFFT_OK;
  TcShape t{};
  if (!make_tc_shape(a, &t)) return fail(SFFT_EPARAM, "tensor-core kernel does not support this shape");
  static uint32_t configured = 0;
  if (t.smem_bytes > configured) {
    cudaError_t e = cudaFuncSetAttribute(k_gate_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kMaxSmem);
    if (e != cudaSuccess) return cuda_fail(e, "tc smem attribute");
    configured = kMaxSmem;
  }
  const uint64_t blocks = a.n * t.mtiles;
  k_gate_tc<<<(unsigned)blocks, kThreads, t.smem_bytes, st>>>(a, t);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SFFT_OK : cuda_fail(e, "tc gate kernel launch");
}

}  // namespace sfft
