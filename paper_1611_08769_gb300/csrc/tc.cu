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
// Two kernels per level:
//  * k_expand_b writes, once per gate, the B operand in its tensor-core form:
//    for every 64-row slice of B' the exact shared-memory image of the
//    128B-swizzled K-major fp16 tile (ndpad byte columns x 64 K values);
//  * k_gate_tc, one CTA (16 warps) per 128-row tile of a gate's output: the
//    A~ tile arrives by one bulk copy (cp.async.bulk + mbarrier transaction
//    count) and is complemented in place when the descriptor asks for P - A;
//    the B slices stream through a shared-memory ring by 1-D bulk copies
//    (already swizzled, no instructions spent on them); per slice the
//    threads expand the A bits into a swizzled fp16 tile (two buffers) and
//    one thread issues the tcgen05.mma chain into the TMEM accumulator and
//    commits to mbarriers that free the A buffer and the ring slot; the
//    epilogue reads the accumulator with tcgen05.ld, takes A~ and the tile's
//    B' rows from shared memory, builds both output tiles in shared memory
//    and writes each back with one bulk store.
// Every mbarrier wait is bounded (~2 s); on timeout the kernel records
// KERR_MMA_TIMEOUT, waits (bounded) for its own MMAs, frees its TMEM and
// returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "common.h"
#include "kargs.h"
#include "plan.h"
#include "rng.h"

namespace sfft {

namespace {

constexpr int kThreads = 512;
constexpr int kTileM = 128;
constexpr int kBK = 64;                        // K elements per slice (128 bytes of fp16)
constexpr uint32_t kSpinLimit = 1u << 26;
constexpr uint64_t kWaitNs = 2000000000ull;    // bound of any single mbarrier wait
constexpr uint32_t kMaxSmem = 232448;          // 227 KB opt-in per CTA
constexpr int kExpandThreads = 256;

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

__device__ __forceinline__ int nib(uint32_t code, int k) {
  return (int)((int32_t)(code << (28 - 4 * k)) >> 28);
}

// Eight bits -> eight fp16 values 1.0 / 0.0 (16 bytes, bit q -> element q).
// y = x * 0x8001 holds x at bit 0 and at bit 15, so bits 2t and 2t+1 of x sit
// at positions 2t and 16 + 2t; masking them and multiplying by 0x3C00 >> 2t
// moves each to its half's 0x3C00 (fp16 1.0) in two instructions per word.
__device__ __forceinline__ uint4 byte_to_h8(uint32_t x) {
  const uint32_t y = x * 0x8001u;
  uint4 v;
  v.x = (y & 0x00010001u) * 0x3C00u;
  v.y = (y & 0x00040004u) * 0x0F00u;
  v.z = (y & 0x00100010u) * 0x03C0u;
  v.w = (y & 0x00400040u) * 0x00F0u;
  return v;
}

__device__ __forceinline__ const uint32_t* ct_ptr(const KArgs& a, uint32_t ref) {
  return a.base[ref >> 30] + (uint64_t)(ref & SLOT_MASK) * a.ctw;
}

}  // namespace

struct TcShape {
  uint32_t nd, ndpad, tmem_cols, mtiles, kblocks, nstages;
  uint32_t n0_len, n1_len;   // MMA N of the two column chunks (n1_len 0 if one chunk)
  uint32_t btile;            // bytes of one expanded B slice (ndpad x 128)
  uint32_t smem_bytes;
};

// ---------------------------------------------------------------------------
// B operand expansion: grid = jobs x kblocks, one swizzled slice image each.
// Job j expands the B operand of gate j (job 0 for every gate when
// a.bx_shared). Output slice (j, kb) lives at a.bx + (j kblocks + kb) btile.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kExpandThreads) k_expand_b(KArgs a, TcShape t) {
  extern __shared__ uint32_t raw[];   // 64 rows x W words
  const uint32_t W = a.W;
  const uint64_t job = blockIdx.x / t.kblocks;
  const uint32_t kb = blockIdx.x % t.kblocks;
  if (job >= a.n) return;
  const uint32_t* B = ct_ptr(a, a.desc[job].b);
  const uint32_t k0 = kb * kBK;
  const uint32_t krows = (a.Ng - k0) < (uint32_t)kBK ? (a.Ng - k0) : (uint32_t)kBK;
  const uint32_t* src = B + (uint64_t)k0 * W;
  for (uint32_t e = threadIdx.x; e < (uint32_t)kBK * W; e += kExpandThreads)
    raw[e] = e < krows * W ? __ldg(src + e) : 0u;
  __syncthreads();
  uint4* dst = (uint4*)(a.bx + (job * t.kblocks + kb) * (uint64_t)t.btile);
  // 16-byte unit u of the tile image: row n = u / 8, stored position p = u % 8
  // holds K chunk c = p ^ (n & 7); digit n = byte (n % 4) of word (n / 4).
  for (uint32_t u = threadIdx.x; u < t.ndpad * 8u; u += kExpandThreads) {
    const uint32_t n = u >> 3, c = (u & 7u) ^ (n & 7u);
    uint4 v = make_uint4(0, 0, 0, 0);
    if (n < t.nd) {
      const uint32_t w = n >> 2, b = n & 3u;
      const uint32_t* rp = raw + c * 8u * W + w;
      const uint32_t sel = b | ((b + 4) << 8);
      v.x = (__byte_perm(rp[0], rp[W], sel) & 0x00FF00FFu) | 0x64006400u;
      v.y = (__byte_perm(rp[2 * W], rp[3 * W], sel) & 0x00FF00FFu) | 0x64006400u;
      v.z = (__byte_perm(rp[4 * W], rp[5 * W], sel) & 0x00FF00FFu) | 0x64006400u;
      v.w = (__byte_perm(rp[6 * W], rp[7 * W], sel) & 0x00FF00FFu) | 0x64006400u;
    }
    dst[u] = v;
  }
}

// ---------------------------------------------------------------------------
// Shared-memory layout of k_gate_tc (offsets from a 1024-aligned base):
//   ring    nstages x btile     expanded B slices (bulk copies)
//   stageA  kAStages x 16 KB    expanded A slices
//   tileA   128 x W words       A~ rows
//   spop    128 words, then 24 mbarriers, the TMEM address slot, a flag
// The epilogue reuses ring slot 0 for the tile's B' rows and slots 1, 2 for
// the two output tiles (each slot >= 128 W words since ndpad >= 4 W).
//
// Warp roles in the main loop (no CTA-wide barrier inside it):
//   warp 0, lane 0   MMA issuer: waits "A stage full" and "B slot full",
//                    issues the MMA chain, commits "A stage free" and
//                    "B slot free"
//   warp 1, lane 0   producer: refills each B slot once its MMAs are done
//   warps 2 .. 15    expand A slices; each warp arrives on "A stage full"
// ---------------------------------------------------------------------------
constexpr uint32_t kAStages = 4;
constexpr uint32_t kExpandWarps = kThreads / 32 - 2;

__global__ void __launch_bounds__(kThreads, 1) k_gate_tc(KArgs a, TcShape t) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t W = a.W, L = a.L, NP1 = W / L;
  uint8_t* ring = smem;
  uint8_t* stageA = ring + t.nstages * t.btile;
  uint32_t* tileA = (uint32_t*)(stageA + kAStages * 16384u);
  uint32_t* spop = tileA + kTileM * W;
  uint64_t* bars = (uint64_t*)(spop + kTileM);
  uint64_t* full = bars;          // [4] B slice landed
  uint64_t* bfree = bars + 4;     // [4] MMAs reading the B slot finished
  uint64_t* afull = bars + 8;     // [4] A stage expanded (one arrival per expander warp)
  uint64_t* afree = bars + 12;    // [4] MMAs reading the A stage finished
  uint64_t* abar = bars + 16;     // A tile landed
  uint64_t* ebar = bars + 17;     // epilogue B rows landed
  uint64_t* done = bars + 18;     // all MMAs finished
  uint32_t* tslot = (uint32_t*)(bars + 24);
  volatile int* sflag = (volatile int*)(tslot + 1);   // a bounded wait ran out

  const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint64_t g = blockIdx.x / t.mtiles;
  const uint32_t row0 = (blockIdx.x % t.mtiles) * kTileM;
  if (g >= a.n) return;
  const uint32_t rows = (a.Ng - row0) < (uint32_t)kTileM ? (a.Ng - row0) : (uint32_t)kTileM;
  const GateDesc d = a.desc[g];
  const GateAux x = a.aux[g];
  const bool gen = (d.a >> 30) == REG_GEN;
  const uint32_t* A = gen ? nullptr : ct_ptr(a, d.a);
  const uint64_t gst = gen ? stream_out(a.gen_state, d.a & SLOT_MASK) : 0;
  const uint32_t* B = ct_ptr(a, d.b);
  const uint8_t* bx = a.bx + (a.bx_shared ? 0 : g) * t.kblocks * (uint64_t)t.btile;
  const bool comp = (x.flags & 1u) != 0;

  if (tid == 0) {
    for (int b = 0; b < 19; b++) mbar_init(&bars[b], (b >= 8 && b < 12) ? kExpandWarps : 1u);
    *sflag = 0;
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
      mbar_expect_tx(&full[s], t.btile);
      bulk_g2s(ring + s * t.btile, bx + (uint64_t)s * t.btile, t.btile, &full[s]);
    }
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
  // Row i of P has one nonzero word: 2^(i % 32) at word (i / ell) L + (i % ell) / 32.
  if (tid < kTileM) {
    const uint32_t r = tid, i = row0 + r;
    const uint32_t pidx = (i / a.ell) * L + (i % a.ell) / 32, pval = 1u << (i % 32);
    uint32_t pc = 0;
    if (comp && r < rows) {
      uint32_t borrow = 0, l = 0;
      for (uint32_t w = 0; w < W; w++) {
        if (l == 0) borrow = 0;
        const uint64_t dv = (uint64_t)(w == pidx ? pval : 0u) - tileA[r * W + w] - borrow;
        const uint32_t v = (uint32_t)dv;
        borrow = (uint32_t)(dv >> 63);
        tileA[r * W + w] = v;
        pc += __popc(v);
        if (++l == L) l = 0;
      }
    } else {
      for (uint32_t w = 0; w < W; w++) pc += __popc(tileA[r * W + w]);
    }
    spop[r] = pc;
  }
  tc_fence_before();
  bool ok = !__syncthreads_or(timed_out);
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (ok) {
    if (warp == 0) {
      // ---------------------------------------------------------- MMA issuer
      if (lane == 0) {
        const uint32_t idesc0 = idesc_f16(kTileM, t.n0_len), idesc1 = idesc_f16(kTileM, t.n1_len);
        for (uint32_t kb = 0; kb < t.kblocks; kb++) {
          const uint32_t s = kb % kAStages, slot = kb % t.nstages;
          if (*sflag || !mbar_wait_bounded(&afull[s], (kb / kAStages) & 1) ||
              !mbar_wait_bounded(&full[slot], (kb / t.nstages) & 1)) {
            *sflag = 1;
            break;
          }
          tc_fence_after();
          const uint32_t a_base = smem_u32(stageA + s * 16384u), b_base = smem_u32(ring + slot * t.btile);
#pragma unroll
          for (uint32_t ks = 0; ks < kBK / 16; ks++) {
            const uint64_t ad = sw128_desc(a_base + ks * 32);
            mma_f16(tmem, ad, sw128_desc(b_base + ks * 32), idesc0, (kb | ks) != 0);
            if (t.n1_len)
              mma_f16(tmem + t.n0_len, ad, sw128_desc(b_base + t.n0_len * 128u + ks * 32), idesc1,
                      (kb | ks) != 0);
          }
          mma_commit(&afree[s]);
          mma_commit(&bfree[slot]);
        }
        mma_commit(done);   // tracks every MMA issued above
      }
    } else if (warp == 1) {
      // ------------------------------------------------------------ producer
      if (lane == 0) {
        for (uint32_t kb = t.nstages; kb < t.kblocks; kb++) {
          const uint32_t slot = kb % t.nstages, prev = kb - t.nstages;
          if (*sflag || !mbar_wait_bounded(&bfree[slot], (prev / t.nstages) & 1)) {
            *sflag = 1;
            break;
          }
          mbar_expect_tx(&full[slot], t.btile);
          bulk_g2s(ring + slot * t.btile, bx + (uint64_t)kb * t.btile, t.btile, &full[slot]);
        }
      }
    } else {
      // ----------------------------------------------------------- expanders
      const uint32_t et = tid - 64;   // 0 .. 32 kExpandWarps - 1
      for (uint32_t kb = 0; kb < t.kblocks; kb++) {
        const uint32_t s = kb % kAStages;
        // lane 0 decides for the whole warp: stop if another role gave up, or
        // once the MMAs of slice kb - kAStages (last readers of this stage) are done
        int stop = 0;
        if (lane == 0) {
          stop = *sflag;
          if (!stop && kb >= kAStages &&
              !mbar_wait_bounded(&afree[s], ((kb - kAStages) / kAStages) & 1)) {
            *sflag = 1;
            stop = 1;
          }
        }
        if (__shfl_sync(0xFFFFFFFFu, stop, 0)) break;
        uint8_t* sA = stageA + s * 16384u;
        for (uint32_t e = et; e < kTileM * 8u; e += 32u * kExpandWarps) {
          const uint32_t r = e >> 3, c = e & 7;
          const uint32_t kbit = kb * kBK + c * 8;
          const uint32_t wi = kbit >> 5;
          const uint32_t byte = wi < W ? (tileA[r * W + wi] >> (kbit & 31)) & 0xFFu : 0u;
          *(uint4*)(sA + sw128_off(r, c)) = byte_to_h8(byte);
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&afull[s])) : "memory");
      }
    }
  }
  __syncthreads();
  if (ok && *sflag) ok = false;
  if (ok) {
    // every MMA finished -> the ring is free: fetch the tile's B' rows (for c2 B)
    bool w_ok = mbar_wait_bounded(done, 0);
    if (w_ok && tid == 0) {
      mbar_expect_tx(ebar, rows * W * 4u);
      bulk_g2s(ring, B + (uint64_t)row0 * W, rows * W * 4u, ebar);
    }
    w_ok = w_ok && mbar_wait_bounded(ebar, 0);
    ok = !__syncthreads_or(!w_ok);
  }
  if (!ok) {
    if (tid == 0 && a.err) atomicExch(a.err, KERR_MMA_TIMEOUT);
    mbar_wait_bounded(done, 0);   // bounded: let own MMAs drain before TMEM is freed
  }
  tc_fence_after();

  if (ok) {
    // Epilogue, phase 1 (all warps): warp w reads TMEM lanes 32 (w % 4) ..
    // (its rows) and every fourth 16-column chunk starting at chunk w / 4;
    // each word's product part K[r][w] = sum_b S[r][4w+b] 2^(8b) goes to
    // shared memory as int64 (ring slots 1-2, free now).
    int64_t* Kv = (int64_t*)(ring + t.btile);
    {
      const uint32_t r = (warp & 3) * 32 + lane;
      const bool live = r < rows;
      const int64_t bias = 1024 * (int64_t)spop[r];
      for (uint32_t n0 = (warp >> 2) * 16u; n0 < t.nd; n0 += 64u) {
        uint32_t v[16];
        tmem_ld16(tmem + (((warp & 3) * 32u) << 16) + n0, v);
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const uint32_t w = n0 / 4 + q;
          if (w >= W || !live) continue;
          int64_t k = 0;
#pragma unroll
          for (int b = 0; b < 4; b++) {
            const int64_t sv = (int64_t)__float2int_rn(__uint_as_float(v[4 * q + b])) - bias;
            k += sv << (8 * b);
          }
          Kv[r * W + w] = k;
        }
      }
    }
    __syncthreads();
    // Phase 2: one thread per (row, element): linear terms and the limb
    // carries of the element; output tile 0 -> stage A area, output tile 1
    // overwrites the tile's B' rows (each word read before it is replaced).
    const uint32_t* Bt = (const uint32_t*)ring;
    uint32_t* T0 = (uint32_t*)stageA;
    uint32_t* T1 = (uint32_t*)ring;
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
    for (uint32_t task = tid; task < kTileM * NP1; task += kThreads) {
      const uint32_t r = task % kTileM, j = task / kTileM, i = row0 + r;
      if (r >= rows) continue;
      const uint32_t pidx = (i / a.ell) * L + (i % a.ell) / 32, pval = 1u << (i % 32);
      int64_t carry0 = 0, carry1 = 0;
      for (uint32_t w = j * L; w < (j + 1) * L; w++) {
        const int64_t k = Kv[r * W + w];
        const int64_t aw = (int64_t)tileA[r * W + w];
        const int64_t bw = (int64_t)Bt[r * W + w];
        const int64_t pw = w == pidx ? (int64_t)pval : 0;
        const int64_t o0 = c03 * k + c01 * aw + c02 * bw + c00 * pw + carry0;
        const int64_t o1 = c13 * k + c11 * aw + c12 * bw + c10 * pw + carry1;
        carry0 = o0 >> 32;
        carry1 = o1 >> 32;
        T0[r * W + w] = (uint32_t)o0;
        T1[r * W + w] = (uint32_t)o1;
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
  if (a.Ng < 128 || a.W == 0) return false;
  t->nd = a.W * 4;
  t->ndpad = (t->nd + 15) / 16 * 16;
  if (t->ndpad > 512) return false;
  t->n0_len = t->ndpad < 256 ? t->ndpad : 256;
  t->n1_len = t->ndpad - t->n0_len;
  t->tmem_cols = 32;
  while (t->tmem_cols < t->ndpad) t->tmem_cols *= 2;
  t->mtiles = (a.Ng + kTileM - 1) / kTileM;
  t->kblocks = (a.Ng + kBK - 1) / kBK;
  t->btile = t->ndpad * 128u;
  for (uint32_t ns = 4; ns >= 3; ns--) {
    const uint32_t bytes = 1024u + ns * t->btile + kAStages * 16384u + (uint32_t)kTileM * a.W * 4u +
                           (uint32_t)kTileM * 4u + 256u;
    if (bytes <= kMaxSmem) {
      t->nstages = ns;
      t->smem_bytes = bytes;
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

uint64_t tc_bx_bytes_per_gate(const KArgs& a) {
  TcShape t;
  if (!make_tc_shape(a, &t)) return 0;
  return (uint64_t)t.kblocks * t.btile;
}

// A level runs in chunks of gates (expand a chunk's B operands, then multiply
// it) so that the expansion buffer stays bounded; the chunk is large enough
// that each GEMM launch spans many waves of CTAs.
constexpr uint64_t kBxL2Budget = 512ull << 20;

uint64_t tc_chunk_gates(const KArgs& a) {
  const uint64_t per = tc_bx_bytes_per_gate(a);
  if (per == 0) return 0;
  const uint64_t c = std::min<uint64_t>(kBxL2Budget / per, 4096);
  return c ? c : 1;
}

uint64_t tc_bx_bytes(const KArgs& a, uint64_t gates) {
  const uint64_t c = tc_chunk_gates(a);
  return (gates < c ? gates : c) * tc_bx_bytes_per_gate(a);
}

int launch_gates_tc(const KArgs& a, cudaStream_t st) {
  if (a.n == 0) return SFFT_OK;
  TcShape t{};
  if (!make_tc_shape(a, &t)) return fail(SFFT_EPARAM, "tensor-core kernel does not support this shape");
  if (!a.bx) return fail(SFFT_EINVAL, "tensor-core kernel needs its B expansion buffer");
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_gate_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kMaxSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_expand_b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
    if (e != cudaSuccess) return cuda_fail(e, "tc smem attribute");
    configured = true;
  }
  const uint64_t chunk = a.bx_shared ? a.n : tc_chunk_gates(a);
  for (uint64_t c0 = 0; c0 < a.n; c0 += chunk) {
    KArgs ca = a;
    ca.desc = a.desc + c0;
    ca.aux = a.aux + c0;
    ca.n = (a.n - c0) < chunk ? (a.n - c0) : chunk;
    KArgs ea = ca;
    ea.n = a.bx_shared ? 1 : ca.n;
    k_expand_b<<<(unsigned)(ea.n * t.kblocks), kExpandThreads, kBK * a.W * 4u, st>>>(ea, t);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "B expansion launch");
    k_gate_tc<<<(unsigned)(ca.n * t.mtiles), kThreads, t.smem_bytes, st>>>(ca, t);
    count_launches(2);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "tc gate kernel launch");
  }
  return SFFT_OK;
}

}  // namespace sfft
