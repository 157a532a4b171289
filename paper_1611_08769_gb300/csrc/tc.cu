// Gate product on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// The GSW product K = BitDecomp(A~) B' (Sec. 7: an N x N matrix product per
// gate) is a dense contraction of a {0,1} matrix with the entries of B'.
// Every ell-bit entry of B' is cut into D = ceil(ell / dw) digits of dw bits
// (dw = 11, or fewer if Ng (2^dw - 1) would reach 2^24), so that per output
// row i and digit column (element e, digit d)
//     S[i][e,d] = sum_k bit_k(A~_i) * digit_d(B'_k[e])  <=  Ng (2^dw - 1)  <  2^24.
// Digits up to 2047 are exact fp16 values and every partial sum is an
// integer below 2^24, so an fp16 x fp16 -> fp32 MMA computes S exactly. The
// epilogue forms K[i][e] = sum_d S[i][e,d] 2^(dw d) (mod 2^ell) word by word
// and adds the linear terms c0 P + c1 A + c2 B with the limb carries of the
// element, exactly as the integer kernel does.
//
// Two kernels per level:
//  * k_expand_b writes, once per gate, the B operand in its tensor-core form:
//    for every 64-row slice of B' the exact shared-memory image of the
//    128B-swizzled K-major fp16 tile (digit columns x 64 K values);
//  * k_gate_tc, one CTA (16 warps) per group of J work items (an item is a
//    128-row tile of one gate's output; J > 1 for small ciphertexts so the
//    CTA's fixed costs are shared): the A~ tiles arrive by bulk copies
//    (cp.async.bulk + mbarrier transaction count) and are complemented in
//    place when the descriptor asks for P - A; the B slices stream through a
//    shared-memory ring by 1-D bulk copies (already swizzled); per (item,
//    slice) step 14 warps expand the A bits into a swizzled fp16 tile and one
//    warp issues the step's tcgen05.mma instructions (one elected lane, the
//    MMAs and their commits in one instruction group) into the item's TMEM
//    accumulator; the commits free the A buffer and the ring slot. The
//    epilogue reads each accumulator with tcgen05.ld (all 16 warps turn digit
//    sums into int64 word sums), then one thread per (row, element) runs the
//    element's carry chain, and both output tiles go back by bulk stores.
// Every mbarrier wait is bounded (~2 s); on timeout the kernel records
// KERR_MMA_TIMEOUT, waits (bounded) for its own MMAs, frees its TMEM and
// returns.
#include <cuda_fp16.h>
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
constexpr uint32_t kMaxDigitBits = 11;         // fp16 holds the integers 0 .. 2048 exactly

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
// iteration cap, whichever comes first). The timer is read only once the
// first probe finds the phase still open.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0; it < kSpinLimit; it++) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 255u && global_ns() - t0 > kWaitNs) return false;
  }
  return false;
}

// As mbar_wait_bounded, and also gives up once `flag` is set (another role
// stopped); the flag is read only on the slow path.
__device__ __forceinline__ bool mbar_wait_flag(uint64_t* bar, uint32_t parity, volatile int* flag) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0; it < kSpinLimit; it++) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 255u && (*flag || global_ns() - t0 > kWaitNs)) return false;
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

// One 64-wide K slice of one item, issued by one elected lane of the calling
// warp (every lane executes the statement; the MMAs and the commits that
// track them sit under the same elect.sync predicate, so one thread issues
// all of them):
//   D[d0] (+)= A * B0^T over four K=16 steps, the same into D[d1] with B1 when
//   `two` is set; then commit -> fb, and -> fd if `last` (one commit per slice:
//   a second one per slice costs the tensor pipe measurably).
// A sits in tensor memory at column `at` (row i in lane i, two fp16 K values
// per 32-bit column: a K=16 step is 8 columns); B0, B1 are 128B-swizzled
// K-major shared-memory tiles (a descriptor advances 32 bytes = 2 units per
// step). `acc` = 0 starts the accumulator (first slice of the item).
__device__ __forceinline__ void mma_slice(uint32_t d0, uint32_t d1, uint32_t at, uint64_t b0,
                                          uint64_t b1, uint32_t id0, uint32_t id1, uint32_t acc,
                                          uint32_t two, uint64_t* fb, uint64_t* fd, uint32_t last) {
  asm volatile(
      "{\n .reg .pred e, e2, e3, p, t;\n .reg .b32 a1, a2, a3;\n .reg .b64 x1, x2, x3, y1, y2, y3;\n"
      " elect.sync _|e, 0xffffffff;\n"
      " setp.ne.b32 p, %8, 0;\n"
      " setp.eq.b32 t, %8, %8;\n"
      " setp.ne.and.b32 e2, %9, 0, e;\n"
      " setp.ne.and.b32 e3, %12, 0, e;\n"
      " add.u32 a1, %3, 8;\n add.u32 a2, %3, 16;\n add.u32 a3, %3, 24;\n"
      " add.u64 x1, %4, 2;\n add.u64 x2, %4, 4;\n add.u64 x3, %4, 6;\n"
      " add.u64 y1, %5, 2;\n add.u64 y2, %5, 4;\n add.u64 y3, %5, 6;\n"
      " @e tcgen05.mma.cta_group::1.kind::f16 [%1], [%3], %4, %6, p;\n"
      " @e tcgen05.mma.cta_group::1.kind::f16 [%1], [a1], x1, %6, t;\n"
      " @e tcgen05.mma.cta_group::1.kind::f16 [%1], [a2], x2, %6, t;\n"
      " @e tcgen05.mma.cta_group::1.kind::f16 [%1], [a3], x3, %6, t;\n"
      " @e2 tcgen05.mma.cta_group::1.kind::f16 [%2], [%3], %5, %7, p;\n"
      " @e2 tcgen05.mma.cta_group::1.kind::f16 [%2], [a1], y1, %7, t;\n"
      " @e2 tcgen05.mma.cta_group::1.kind::f16 [%2], [a2], y2, %7, t;\n"
      " @e2 tcgen05.mma.cta_group::1.kind::f16 [%2], [a3], y3, %7, t;\n"
      " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%10];\n"
      " @e3 tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%11];\n}\n" ::"r"(0u),
      "r"(d0), "r"(d1), "r"(at), "l"(b0), "l"(b1), "r"(id0), "r"(id1), "r"(acc), "r"(two),
      "r"(smem_u32(fb)), "r"(smem_u32(fd)), "r"(last)
      : "memory");
}

// Commit -> bar from the elected lane of the calling warp (the lane that
// issued the warp's MMAs: with every lane active, elect.sync picks the same
// leader each time).
__device__ __forceinline__ void mma_commit_elected(uint64_t* bar) {
  asm volatile(
      "{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n"
      " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n" ::"r"(
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

// Each thread stores 32 consecutive 32-bit columns of its own lane.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]),
      "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]),
      "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]),
      "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
      : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
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

__host__ __device__ constexpr uint32_t idesc_f16(uint32_t M, uint32_t N) {
  return (1u << 4) | ((N >> 3) << 17) | ((M >> 4) << 24);
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
  uint32_t dw;               // digit width in bits
  uint32_t D, dpad;          // digits per element, digit columns per element (multiple of 16)
  uint32_t ndpad;            // digit columns of a row (elements x dpad)
  uint32_t tmem_cols, mtiles, kblocks, nstages;
  uint32_t n0_len, n1_len;   // MMA N of the two column chunks (n1_len 0 if one chunk)
  uint32_t btile;            // bytes of one expanded B slice (ndpad x 128)
  uint32_t items;            // work items (gate x 128-row tile) per CTA
  uint32_t smem_bytes;
};

// ---------------------------------------------------------------------------
// B operand expansion: grid = jobs x kblocks, one swizzled slice image each.
// Job j expands the B operand of gate j (job 0 for every gate when
// a.bx_shared). Output slice (j, kb) lives at a.bx + (j kblocks + kb) btile.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kExpandThreads) k_expand_b(KArgs a, TcShape t) {
  extern __shared__ uint32_t raw[];   // 64 rows x W words
  const uint32_t W = a.W, L = a.L;
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
  const uint32_t mask = (1u << t.dw) - 1u;
  // 16-byte unit u of the tile image: row n = u / 8, stored position p = u % 8
  // holds K chunk c = p ^ (n & 7); row n is digit d = n % dpad of element
  // e = n / dpad: bits dw d .. dw d + dw - 1 of the element (zero past ell).
  for (uint32_t u = threadIdx.x; u < t.ndpad * 8u; u += kExpandThreads) {
    const uint32_t n = u >> 3, c = (u & 7u) ^ (n & 7u);
    const uint32_t e = n / t.dpad, d = n - e * t.dpad;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (d < t.D) {
      const uint32_t bit = d * t.dw, wl = bit >> 5, sh = bit & 31u;
      const bool hi = wl + 1 < L;   // the digit may continue in the element's next limb
      const uint32_t* rp = raw + c * 8u * W + e * L + wl;
      uint32_t h[8];
#pragma unroll
      for (int q = 0; q < 8; q++) {
        const uint32_t dig = __funnelshift_r(rp[q * W], hi ? rp[q * W + 1] : 0u, sh) & mask;
        h[q] = __half_as_ushort(__uint2half_rn(dig));
      }
      v.x = h[0] | (h[1] << 16);
      v.y = h[2] | (h[3] << 16);
      v.z = h[4] | (h[5] << 16);
      v.w = h[6] | (h[7] << 16);
    }
    dst[u] = v;
  }
}


// ---------------------------------------------------------------------------
// Shared-memory layout of k_gate_tc (offsets from a 1024-aligned base), for J
// work items per CTA (an item = one gate's 128-row output tile):
//   ring    nstages x btile       expanded B slices (bulk copies)
//   tileA   J x 128 x W words     A~ rows of every item
//   brows   J x 128 x W words     B' rows of every item (epilogue)
//   then 27 mbarriers, the TMEM address slot, a flag, and from the 32nd
//   8-byte word on 4 words per item (gate, row0, rows, K rotation)
// Tensor memory (512 columns): item j's accumulator at columns j ndpad ..
// (j+1) ndpad - 1; the kAStages expanded A slices (32 columns each: 64 fp16
// K values per lane = row) in the last 32 kAStages columns.
// Epilogue (after the main loop): the ring holds the int64 word sums of the
// current item (1024 (W | 1) bytes); output tiles 0 and 1 overwrite the
// item's A~ and B' rows in place.
//
// Warp roles in the main loop (no CTA-wide barrier inside it); the loop runs
// over steps = (item, 64-wide K slice), J x kblocks of them. Step st uses B
// slot st % nstages and A stage st % kAStages; one pair of barriers per slot:
// full[slot] completes when the slice's B bytes landed (transaction count of
// the producer's arrival) and the four expander warps of the step arrived;
// bfree[slot] when the step's MMAs are done (their single commit).
//   warp 0           MMA issuer (one elected lane issues, the warp runs the
//                    loop): waits full, issues the slice's MMAs into the
//                    item's TMEM columns, commits -> bfree
//   warp 1, lane 0   producer: refills a B slot once the MMAs of its
//                    previous step are done
//   warps 4 .. 11    expanders, two groups of four warps (one warp per TMEM
//                    lane quarter) taking alternate steps: once the MMAs of
//                    step st - kAStages (the stage's last readers) are done,
//                    each thread turns its row's 64 bits of the slice into 64
//                    fp16 values and stores them to its lane of the stage's
//                    columns; each warp arrives on full. (nstages >= kAStages
//                    keeps these waits unambiguous: the next phase of the
//                    slot needs this step's MMAs first.)
// ---------------------------------------------------------------------------
constexpr uint32_t kAStages = 4;
constexpr uint32_t kExpandGroups = 2;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kAColumns = 32 * kAStages;   // tensor-memory columns of the A stages

// Position of a main-loop step: B slot and the parity of its phase, item and
// K slice. Advanced incrementally, so the per-step paths divide nothing.
struct StepPos {
  uint32_t slot, phase, j, kb;
  __device__ __forceinline__ void start(uint32_t st, const TcShape& t) {
    slot = st % t.nstages;
    phase = (st / t.nstages) & 1u;
    j = st / t.kblocks;
    kb = st % t.kblocks;
  }
  __device__ __forceinline__ void next(const TcShape& t) {
    if (++slot == t.nstages) {
      slot = 0;
      phase ^= 1u;
    }
    if (++kb == t.kblocks) {
      kb = 0;
      j++;
    }
  }
};

__global__ void __launch_bounds__(kThreads, 1) k_gate_tc(KArgs a, TcShape t) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t W = a.W, L = a.L, NP1 = W / L, J = t.items;
  uint8_t* ring = smem;
  uint32_t* tileA = (uint32_t*)(ring + t.nstages * t.btile);
  uint32_t* brows = tileA + J * kTileM * W;
  uint64_t* bars = (uint64_t*)(brows + J * kTileM * W);
  uint64_t* full = bars;          // [8] B slice landed and A stage expanded
  uint64_t* bfree = bars + 8;     // [8] MMAs of the slot's step finished
  uint64_t* abar = bars + 24;     // A tiles landed
  uint64_t* ebar = bars + 25;     // epilogue B rows landed
  uint64_t* done = bars + 26;     // all MMAs finished
  uint32_t* tslot = (uint32_t*)(bars + 28);
  volatile int* sflag = (volatile int*)(tslot + 1);   // a bounded wait ran out

  const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint64_t n_items = a.n * t.mtiles;
  const uint64_t item0 = (uint64_t)blockIdx.x * J;
  if (item0 >= n_items) return;
  const uint32_t nj = (uint32_t)((n_items - item0) < J ? (n_items - item0) : J);  // live items
  const uint32_t steps = nj * t.kblocks;
  // item j: gate, first row, live rows (computed once, kept in shared memory)
  // The K slices of an item run in rotated order (tile m starts at slice
  // m kblocks / mtiles; the exact integer sums do not depend on the order), so
  // the tiles of one gate stream different B slices at any moment.
  uint32_t* iinfo = (uint32_t*)(bars + 32);   // [J][4]: gate, row0, rows, rotation
  if (tid < nj) {
    const uint64_t it = item0 + tid;
    const uint32_t m = (uint32_t)(it % t.mtiles), r0 = m * kTileM;
    iinfo[4 * tid] = (uint32_t)(it / t.mtiles);
    iinfo[4 * tid + 1] = r0;
    iinfo[4 * tid + 2] = (a.Ng - r0) < (uint32_t)kTileM ? (a.Ng - r0) : (uint32_t)kTileM;
    iinfo[4 * tid + 3] = m * t.kblocks / t.mtiles;
  }
  auto item_gate = [&](uint32_t j) { return (uint64_t)iinfo[4 * j]; };
  auto item_row0 = [&](uint32_t j) { return iinfo[4 * j + 1]; };
  auto item_rows = [&](uint32_t j) { return iinfo[4 * j + 2]; };
  // slice of K consumed by step st (item st / kblocks)
  auto step_kb = [&](uint32_t st) {
    const uint32_t kb = st % t.kblocks + iinfo[4 * (st / t.kblocks) + 3];
    return kb < t.kblocks ? kb : kb - t.kblocks;
  };
  auto item_bx = [&](uint32_t j) {
    return a.bx + (a.bx_shared ? 0 : item_gate(j)) * t.kblocks * (uint64_t)t.btile;
  };

  if (tid == 0) {
    for (int b = 0; b < 27; b++) mbar_init(&bars[b], b < 8 ? 5u : 1u);   // full: producer + 4 warps
    *sflag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(tslot, kTmemCols);
  __syncthreads();
  const bool gen = (a.desc[item_gate(0)].a >> 30) == REG_GEN;   // encryption: every item generated
  if (tid == 0) {
    uint32_t bytes = 0;
    for (uint32_t j = 0; j < nj; j++) bytes += item_rows(j) * W * 4u;
    if (!gen) {
      mbar_expect_tx(abar, bytes);
      for (uint32_t j = 0; j < nj; j++) {
        const uint32_t* A = ct_ptr(a, a.desc[item_gate(j)].a);
        bulk_g2s(tileA + j * kTileM * W, A + (uint64_t)item_row0(j) * W, item_rows(j) * W * 4u, abar);
      }
    }
    // the epilogue's B' rows (for c2 B) arrive during the main loop
    mbar_expect_tx(ebar, bytes);
    for (uint32_t j = 0; j < nj; j++)
      bulk_g2s(brows + j * kTileM * W, ct_ptr(a, a.desc[item_gate(j)].b) + (uint64_t)item_row0(j) * W,
               item_rows(j) * W * 4u, ebar);
    for (uint32_t s = 0; s < t.nstages && s < steps; s++) {
      mbar_expect_tx(&full[s], t.btile);
      bulk_g2s(ring + s * t.btile, item_bx(s / t.kblocks) + (uint64_t)step_kb(s) * t.btile,
               t.btile, &full[s]);
    }
  }
  bool timed_out = false;
  if (gen) {
    for (uint32_t e = tid; e < nj * kTileM * W; e += kThreads) {
      const uint32_t j = e / (kTileM * W), r = (e / W) % kTileM, w = e % W;
      const uint64_t gst = stream_out(a.gen_state, a.desc[item_gate(j)].a & SLOT_MASK);
      tileA[e] = r < item_rows(j) ? r_word(gst, (uint64_t)(item_row0(j) + r) * W + w) : 0u;
    }
  } else {
    timed_out = !mbar_wait_bounded(abar, 0);
    for (uint32_t j = 0; j < nj; j++)   // rows past the last ciphertext row of a partial tile
      for (uint32_t e = item_rows(j) * W + tid; e < kTileM * W; e += kThreads)
        tileA[j * kTileM * W + e] = 0;
  }
  __syncthreads();
  // Complement (P - A) row by row with the borrow chain of each element.
  // Row i of P has one nonzero word: 2^(i % 32) at word (i / ell) L + (i % ell) / 32.
  for (uint32_t task = tid; task < nj * kTileM; task += kThreads) {
    const uint32_t j = task / kTileM, r = task % kTileM, i = item_row0(j) + r;
    if (!(a.aux[item_gate(j)].flags & 1u) || r >= item_rows(j)) continue;
    uint32_t* row = tileA + (j * kTileM + r) * W;
    const uint32_t pidx = (i / a.ell) * L + (i % a.ell) / 32, pval = 1u << (i % 32);
    uint32_t borrow = 0, l = 0;
    for (uint32_t w = 0; w < W; w++) {
      if (l == 0) borrow = 0;
      const uint64_t dv = (uint64_t)(w == pidx ? pval : 0u) - row[w] - borrow;
      row[w] = (uint32_t)dv;
      borrow = (uint32_t)(dv >> 63);
      if (++l == L) l = 0;
    }
  }
  tc_fence_before();
  bool ok = !__syncthreads_or(timed_out);
  tc_fence_after();
  const uint32_t tmem = *tslot;

  if (ok) {
    if (warp == 0) {
      // ---------------------------------------------------------- MMA issuer
      const uint32_t idesc0 = idesc_f16(kTileM, t.n0_len), idesc1 = idesc_f16(kTileM, t.n1_len);
      const uint32_t two = t.n1_len != 0, ring_s = smem_u32(ring);
      const uint32_t acol = tmem + (kTmemCols - kAColumns);
      bool issued_all = true;
      StepPos p;
      p.start(0, t);
      for (uint32_t st = 0; st < steps; st++) {
        if (!__all_sync(0xFFFFFFFFu, mbar_wait_flag(&full[p.slot], p.phase, sflag))) {
          if (lane == 0) *sflag = 1;
          issued_all = false;
          break;
        }
        tc_fence_after();
        const uint32_t b_base = ring_s + p.slot * t.btile;
        const uint32_t d = tmem + p.j * t.ndpad;
        mma_slice(d, d + t.n0_len, acol + 32u * (st & (kAStages - 1)), sw128_desc(b_base),
                  sw128_desc(b_base + t.n0_len * 128u), idesc0, idesc1, p.kb != 0, two, &bfree[p.slot],
                  done, st + 1 == steps);
        p.next(t);
      }
      // after a failed wait, `done` still has to track the MMAs issued so far
      if (!issued_all) mma_commit_elected(done);
    } else if (warp == 1) {
      // ------------------------------------------------------------ producer
      if (lane == 0 && steps > t.nstages) {
        StepPos p;
        p.start(t.nstages, t);
        uint32_t rot = iinfo[4 * p.j + 3];
        const uint8_t* bx = item_bx(p.j);
        for (uint32_t st = t.nstages; st < steps; st++) {
          // the slot's previous step (st - nstages) ran in the other phase
          if (!mbar_wait_flag(&bfree[p.slot], p.phase ^ 1u, sflag)) {
            *sflag = 1;
            break;
          }
          uint32_t kbr = p.kb + rot;
          if (kbr >= t.kblocks) kbr -= t.kblocks;
          mbar_expect_tx(&full[p.slot], t.btile);
          bulk_g2s(ring + p.slot * t.btile, bx + (uint64_t)kbr * t.btile, t.btile, &full[p.slot]);
          const uint32_t oj = p.j;
          p.next(t);
          if (p.j != oj && p.j < nj) {
            rot = iinfo[4 * p.j + 3];
            bx = item_bx(p.j);
          }
        }
      }
    } else if (warp >= 4 && warp < 4 + 4 * kExpandGroups) {
      // ----------------------------------------------------------- expanders
      const uint32_t grp = (warp - 4) / 4, q = warp & 3, r = q * 32 + lane;
      const uint32_t acol = tmem + ((q * 32u) << 16) + (kTmemCols - kAColumns);
      StepPos p;
      p.start(grp, t);
      uint32_t rot = p.j < nj ? iinfo[4 * p.j + 3] : 0u;
      for (uint32_t st = grp; st < steps; st += kExpandGroups) {
        // lane 0 decides for the whole warp: go on once the MMAs of step
        // st - kAStages (the stage's last readers) are done; that step used
        // slot - kAStages, in the previous phase if the slot index wrapped
        int stop = 0;
        if (lane == 0 && st >= kAStages) {
          const bool wrap = p.slot < kAStages;
          const uint32_t ps = wrap ? p.slot + t.nstages - kAStages : p.slot - kAStages;
          if (!mbar_wait_flag(&bfree[ps], wrap ? p.phase ^ 1u : p.phase, sflag)) {
            *sflag = 1;
            stop = 1;
          }
        }
        if (__shfl_sync(0xFFFFFFFFu, stop, 0)) break;
        tc_fence_after();
        uint32_t kb = p.kb + rot;
        if (kb >= t.kblocks) kb -= t.kblocks;
        // row r's bits 64 kb .. 64 kb + 63 (words 2 kb, 2 kb + 1; zero past the
        // row) -> 64 fp16 values, K value k in half k % 2 of column k / 2
        const uint32_t* row = tileA + (p.j * kTileM + r) * W;
        const uint32_t w0 = 2u * kb < W ? row[2u * kb] : 0u;
        const uint32_t w1 = 2u * kb + 1u < W ? row[2u * kb + 1u] : 0u;
        uint32_t v[32];
#pragma unroll
        for (uint32_t b = 0; b < 8; b++) {
          const uint4 h = byte_to_h8(((b < 4 ? w0 : w1) >> (8u * (b & 3u))) & 0xFFu);
          v[4 * b] = h.x;
          v[4 * b + 1] = h.y;
          v[4 * b + 2] = h.z;
          v[4 * b + 3] = h.w;
        }
        tmem_st32(acol + 32u * (st & (kAStages - 1)), v);
        tc_fence_before();
        __syncwarp();
        if (lane == 0)
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&full[p.slot])) : "memory");
        const uint32_t oj = p.j;
        for (uint32_t k = 0; k < kExpandGroups; k++) p.next(t);
        if (p.j != oj && p.j < nj) rot = iinfo[4 * p.j + 3];
      }
    }
  }
  __syncthreads();
  if (ok && *sflag) ok = false;
  if (ok) {
    // every MMA finished and the B' rows landed
    const bool w_ok = mbar_wait_bounded(done, 0) && mbar_wait_bounded(ebar, 0);
    ok = !__syncthreads_or(!w_ok);
  }
  if (!ok) {
    if (tid == 0 && a.err) atomicExch(a.err, KERR_MMA_TIMEOUT);
    mbar_wait_bounded(done, 0);   // bounded: let own MMAs drain before TMEM is freed
    mbar_wait_bounded(ebar, 0);   // and the bulk copies into shared memory
  }
  tc_fence_after();

  // Epilogue. Phase 1 (all warps): warp w reads TMEM lanes 32 (w % 4) .. +31
  // (its rows) over the digit columns of the row's words [w/4 W/4, (w/4+1) W/4);
  // digit d of element e adds S << (dw d mod 32) to word (dw d) / 32 of the
  // element (every word gets at least two digits, in column order) and the
  // int64 word sums go to Kv (row stride KS = W | 1 words of 8 bytes, odd, so
  // a warp's rows fall in distinct bank pairs). Phase 2: one thread per (row,
  // element) runs the element's carry chain with the linear terms; output
  // tile 0 overwrites the item's A~ rows and tile 1 its B' rows in place.
  int64_t* Kv = (int64_t*)ring;
  const uint32_t KS = W | 1u;
  for (uint32_t j = 0; ok && j < nj; j++) {
    const uint64_t g = item_gate(j);
    const uint32_t row0 = item_row0(j), rows = item_rows(j);
    const GateDesc gd = a.desc[g];
    const GateAux x = a.aux[g];
    uint32_t* At = tileA + j * kTileM * W;               // A~ rows, then output tile 0
    uint32_t* Bt = brows + j * kTileM * W;               // B' rows, then output tile 1
    {
      const uint32_t q = warp & 3, cg = warp >> 2, r = q * 32 + lane;
      const uint32_t gw0 = cg * W / 4, gw1 = (cg + 1) * W / 4;
      // first digit column of global word gw (element gw / L, local word gw % L)
      auto first_col = [&](uint32_t gw) {
        const uint32_t e = gw / L, wl = gw - e * L;
        return e * t.dpad + (32u * wl + t.dw - 1) / t.dw;
      };
      if (gw0 < gw1) {
        const uint32_t n0 = first_col(gw0), n1 = first_col(gw1);
        const uint32_t taddr = tmem + ((q * 32u) << 16) + j * t.ndpad;
        int64_t acc = 0;
        uint32_t cur = gw0;
        for (uint32_t c0 = n0 & ~15u; c0 < n1; c0 += 16) {
          uint32_t v[16];
          tmem_ld16(taddr + c0, v);
          const uint32_t e = c0 / t.dpad, dbase = c0 - e * t.dpad;   // a chunk lies in one element
#pragma unroll
          for (uint32_t k = 0; k < 16; k++) {
            const uint32_t n = c0 + k, d = dbase + k;
            if (n >= n0 && n < n1 && d < t.D) {
              const uint32_t bit = d * t.dw, gw = e * L + (bit >> 5);
              if (gw != cur) {
                Kv[r * KS + cur] = acc;
                acc = 0;
                cur = gw;
              }
              acc += (int64_t)__float2int_rn(__uint_as_float(v[k])) << (bit & 31u);
            }
          }
        }
        Kv[r * KS + cur] = acc;   // word gw1 - 1
      }
    }
    __syncthreads();
    {
      const uint32_t code0 = x.code & 0xFFFFu, code1 = x.code >> 16;
      int c00 = nib(code0, 0), c01 = nib(code0, 1), c02 = nib(code0, 2), c03 = nib(code0, 3);
      int c10 = nib(code1, 0), c11 = nib(code1, 1), c12 = nib(code1, 2), c13 = nib(code1, 3);
      if (x.flags & 1u) {  // the stored A is P - A~: c1 A = c1 P - c1 A~
        c00 += c01;
        c01 = -c01;
        c10 += c11;
        c11 = -c11;
      }
      for (uint32_t task = tid; task < kTileM * NP1; task += kThreads) {
        const uint32_t r = task % kTileM, e = task / kTileM, i = row0 + r;
        if (r >= rows) continue;
        // row i of P: 2^(i % 32) at word (i / ell) L + (i % ell) / 32
        const uint32_t pw_at = (i / a.ell) * L + (i % a.ell) / 32;
        const int64_t pval = (int64_t)1 << (i % 32);
        uint32_t* Ar = At + r * W;
        uint32_t* Br = Bt + r * W;
        const int64_t* Kr = Kv + r * KS;
        int64_t carry0 = 0, carry1 = 0;
        for (uint32_t w = e * L; w < (e + 1) * L; w++) {
          const int64_t k = Kr[w], aw = Ar[w], bw = Br[w], pw = w == pw_at ? pval : 0;
          const int64_t o0 = c03 * k + c01 * aw + c02 * bw + c00 * pw + carry0;
          const int64_t o1 = c13 * k + c11 * aw + c12 * bw + c10 * pw + carry1;
          carry0 = o0 >> 32;
          carry1 = o1 >> 32;
          Ar[w] = (uint32_t)o0;
          Br[w] = (uint32_t)o1;
        }
      }
    }
    fence_proxy_async_smem();
    __syncthreads();   // also: Kv is rewritten by the next item's phase 1
    if (tid == 0) {
      if (gd.o0 != REF_NONE)
        bulk_s2g(a.base[gd.o0 >> 30] + (uint64_t)(gd.o0 & SLOT_MASK) * a.ctw + (uint64_t)row0 * W, At,
                 rows * W * 4u);
      if (gd.o1 != REF_NONE)
        bulk_s2g(a.base[gd.o1 >> 30] + (uint64_t)(gd.o1 & SLOT_MASK) * a.ctw + (uint64_t)row0 * W, Bt,
                 rows * W * 4u);
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    }
  }
  // the output tiles stay untouched until the CTA ends: one wait for every store
  if (tid == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

namespace {

uint32_t tc_smem_bytes(uint32_t W, uint32_t btile, uint32_t ns, uint32_t J) {
  return 1024u + ns * btile + 2u * J * (uint32_t)kTileM * W * 4u + 256u + 16u * J;
}

// Shape of the kernel for up to `jmax` items per CTA (0 = the largest that fits).
bool make_tc_shape(const KArgs& a, TcShape* t, uint32_t jmax = 1) {
  if (a.Ng < 128 || a.W == 0 || a.L == 0 || a.ell != 32 * a.L) return false;
  const uint32_t NP1 = a.W / a.L;
  // digit width: exact fp16 operand and every column sum below 2^24
  t->dw = kMaxDigitBits;
  while (t->dw > 1 && (uint64_t)a.Ng * ((1u << t->dw) - 1u) >= (1u << 24)) t->dw--;
  t->D = (a.ell + t->dw - 1) / t->dw;
  t->dpad = (t->D + 15) / 16 * 16;
  t->ndpad = NP1 * t->dpad;
  if (t->ndpad > 512) return false;
  // one MMA up to N = 256, else two balanced chunks (multiples of 16)
  t->n0_len = t->ndpad <= 256 ? t->ndpad : (t->ndpad / 2 + 15) / 16 * 16;
  t->n1_len = t->ndpad - t->n0_len;
  t->mtiles = (a.Ng + kTileM - 1) / kTileM;
  t->kblocks = (a.Ng + kBK - 1) / kBK;
  t->btile = t->ndpad * 128u;
  t->nstages = 0;
  for (uint32_t ns = 8; ns >= kAStages; ns--)
    if (tc_smem_bytes(a.W, t->btile, ns, 1) <= kMaxSmem) {
      t->nstages = ns;
      break;
    }
  // the epilogue keeps the int64 word sums (128 rows of W | 1) in the ring
  if (!t->nstages || t->nstages * t->btile < 1024u * (a.W | 1u)) return false;
  // items per CTA: TMEM columns, stage A room for the epilogue's B rows, smem
  uint32_t J = 1;
  const uint32_t cap = jmax ? jmax : 64;
  if (t->ndpad + kAColumns > kTmemCols) return false;
  while (J < cap && (J + 1) * t->ndpad + kAColumns <= kTmemCols &&
         tc_smem_bytes(a.W, t->btile, t->nstages, J + 1) <= kMaxSmem)
    J++;
  t->items = J;
  t->tmem_cols = kTmemCols;
  t->smem_bytes = tc_smem_bytes(a.W, t->btile, t->nstages, J);
  return true;
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

uint32_t tc_digit_columns(const KArgs& a) {
  TcShape t;
  if (!make_tc_shape(a, &t)) return 0;
  return (a.W / a.L) * t.D;
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
  TcShape t0{};
  if (!make_tc_shape(a, &t0, 0)) return fail(SFFT_EPARAM, "tensor-core kernel does not support this shape");
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
    k_expand_b<<<(unsigned)(ea.n * t0.kblocks), kExpandThreads, kBK * a.W * 4u, st>>>(ea, t0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "B expansion launch");
    // items per CTA: as many as fit, but keep at least two CTAs per SM's worth of work
    const uint64_t items = ca.n * t0.mtiles;
    const uint64_t want = std::max<uint64_t>(1, items / (2 * 152));
    TcShape t{};
    make_tc_shape(a, &t, (uint32_t)std::min<uint64_t>(want, t0.items));
    const uint64_t blocks = (items + t.items - 1) / t.items;
    k_gate_tc<<<(unsigned)blocks, kThreads, t.smem_bytes, st>>>(ca, t);
    count_launches(2);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "tc gate kernel launch");
  }
  return SFFT_OK;
}

}  // namespace sfft
