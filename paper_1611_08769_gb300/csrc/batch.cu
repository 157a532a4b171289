// Batched evaluation: many FFT requests' circuit levels merged into one
// program, optionally replayed as a CUDA graph.
//
// Level l of the merged program holds every request's products of
// multiplicative depth l (all independent), so one launch covers them all;
// wire references are shifted into per-request ranges of one input buffer,
// one output buffer and one scratch pool. GSW leveled evaluation needs no
// evaluation key, so requests encrypted under different client keys batch
// freely as long as (n, ell) agree. The captured graph holds the whole
// sequence of level launches (gate-kernel pairs in L2-sized chunks, then the
// output fix-ups) for fixed buffer pointers and stream; it is re-captured
// when any of them changes.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cstring>
#include <memory>
#include <string>
#include <unordered_map>
#include <vector>

#include "common.h"
#include "netlist.h"
#include "plan.h"

namespace sfft {

namespace {

uint32_t shift_ref(uint32_t ref, const uint64_t off[4]) {
  if (ref == REF_NONE) return ref;
  const uint32_t region = ref >> 30;
  return make_ref(region, (uint32_t)((ref & SLOT_MASK) + off[region]));
}

}  // namespace

// Merges per-request programs level by level. off[r][region] is the first
// slot of request r in each region (scratch / input / output).
void merge_programs(const std::vector<Program>& parts, const std::vector<std::array<uint64_t, 4>>& off,
                    Program* out) {
  size_t levels = 0;
  for (const Program& p : parts) levels = std::max(levels, p.level_off.size() - 1);
  out->desc.clear();
  out->aux.clear();
  out->fix.clear();
  out->level_off.assign(1, 0);
  out->lin_start.clear();
  out->max_width = 0;
  out->products = 0;
  out->noise_ok = true;
  out->noise_bits = 0;
  for (size_t l = 0; l < levels; l++) {
    // every request's products of level l, then every request's linear gates
    const uint64_t before = out->desc.size();
    for (int phase = 0; phase < 2; phase++) {
      if (phase == 1) out->lin_start.push_back(out->desc.size());
      for (size_t r = 0; r < parts.size(); r++) {
        const Program& p = parts[r];
        if (l + 1 >= p.level_off.size()) continue;
        const uint64_t g0 = phase ? p.lin_start[l] : p.level_off[l];
        const uint64_t g1 = phase ? p.level_off[l + 1] : p.lin_start[l];
        for (uint64_t g = g0; g < g1; g++) {
          GateDesc d = p.desc[g];
          d.a = shift_ref(d.a, off[r].data());
          d.b = shift_ref(d.b, off[r].data());
          d.o0 = shift_ref(d.o0, off[r].data());
          d.o1 = shift_ref(d.o1, off[r].data());
          out->desc.push_back(d);
          out->aux.push_back(p.aux[g]);
        }
      }
    }
    const uint64_t width = out->lin_start.back() - before;
    out->level_off.push_back(out->desc.size());
    out->max_width = std::max<uint64_t>(out->max_width, width);
    out->products += width;
  }
  for (size_t r = 0; r < parts.size(); r++) {
    for (FixDesc f : parts[r].fix) {
      f.dst = (uint32_t)(f.dst + off[r][REG_OUT]);
      if (f.kind <= 1) f.src = shift_ref(f.src, off[r].data());
      out->fix.push_back(f);
    }
    out->noise_ok = out->noise_ok && parts[r].noise_ok;
    out->noise_bits = std::max(out->noise_bits, parts[r].noise_bits);
  }
}

// Graph replays of run_program for fixed pointers and stream: two entries
// (the two buffer sets of a double-buffered pipeline), least recently used
// replaced.
struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  const void* key[4] = {nullptr, nullptr, nullptr, nullptr};
  uint64_t bytes = 0, used = 0;
};
struct GraphCache {
  GraphEntry e[2];
  uint64_t clock = 0;
  ~GraphCache() {
    for (GraphEntry& g : e)
      if (g.exec) cudaGraphExecDestroy(g.exec);
  }
};

// Persistent form, per run: the epoch advances (gate flags of earlier runs stay
// behind it), the claim counter and the per-level counts restart.
// Before each persistent run: the next epoch, the claim counter and the level
// counts restarted. Gates compare their producers' flags with the epoch, so a
// wrap of the 32-bit epoch would make old flags look current: at the wrap the
// flags are cleared and the epoch restarts at 1 (once in 2^32 runs).
__global__ void k_persist_begin(uint32_t* epoch, uint32_t* claim, unsigned long long* ldone, uint32_t levels,
                                uint32_t* gflag, uint64_t n) {
  const uint32_t e = *epoch;
  __syncthreads();   // every thread has read the old epoch
  if (e == 0xFFFFFFFFu)
    for (uint64_t g = threadIdx.x; g < n; g += blockDim.x) gflag[g] = 0u;
  if (threadIdx.x == 0) {
    *epoch = e == 0xFFFFFFFFu ? 1u : e + 1u;
    *claim = 0u;
  }
  for (uint32_t l = threadIdx.x; l < levels; l += blockDim.x) ldone[l] = 0ull;
}

// Device state of the persistent form (sfft_batch with SFFT_BATCH_PERSISTENT).
struct PersistState {
  uint32_t* glev = nullptr;       // level of every gate
  GateDeps* gdep = nullptr;       // the gates that produced its A and B (0xFFFFFFFF: an input)
  uint32_t* lwidth = nullptr;     // gates per level
  unsigned long long* ldone = nullptr;
  uint32_t* gflag = nullptr;
  uint32_t* claim = nullptr;
  uint32_t* epoch = nullptr;
  uint32_t levels = 0;
  ~PersistState() {
    cudaFree(glev);
    cudaFree(gdep);
    cudaFree(lwidth);
    cudaFree(ldone);
    cudaFree(gflag);
    cudaFree(claim);
    cudaFree(epoch);
  }
};

// Every product of the program in one launch of the small-ciphertext kernel
// (gates claimed in program order, levels overlapping by one), then the
// output fix-ups.
int run_persistent(const Shape& s, const DeviceProgram& dp, const PersistState& ps, const uint32_t* d_in,
                   uint32_t* d_out, uint32_t* d_scratch, uint64_t scratch_bytes, cudaStream_t st,
                   Timer* tm) {
  if (!d_in || !d_out) return fail(SFFT_EINVAL, "null buffer");
  if (scratch_bytes < dp.scratch_bytes || (dp.scratch_bytes && !d_scratch))
    return fail(SFFT_EINVAL, "scratch buffer too small");
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != dp.device)
    return fail(SFFT_EINVAL, "the current CUDA device is not the one the batch was created on");
  k_persist_begin<<<1, 256, 0, st>>>(ps.epoch, ps.claim, ps.ldone, ps.levels, ps.gflag, dp.level_off.back());
  count_launches(1);
  KArgs a = make_args(s);
  a.base[REG_SCRATCH] = d_scratch;
  a.base[REG_IN] = const_cast<uint32_t*>(d_in);
  a.base[REG_OUT] = d_out;
  a.err = dp.err;
  a.kernel = KERNEL_SM;
  a.desc = dp.desc;
  a.aux = dp.aux;
  a.n = dp.level_off.back();
  a.glev = ps.glev;
  a.gdep = ps.gdep;
  a.lwidth = ps.lwidth;
  a.ldone = ps.ldone;
  a.gflag = ps.gflag;
  a.claim = ps.claim;
  a.epoch = ps.epoch;
  const bool timed = tm && tm->on && a.n;
  a.timer = timed ? tm : nullptr;
  int rc = launch_gates(a, st);
  if (rc) return rc;
  if (timed) {
    tm->launches++;
    tm->products += a.n;
  }
  a.timer = nullptr;
  return launch_fixups(dp.fix, dp.n_fix, a, st);
}

int run_graph(GraphCache* cache, const Shape& s, const DeviceProgram& dp, const PersistState* ps,
              const uint32_t* d_in, uint32_t* d_out, uint32_t* d_scratch, uint64_t scratch_bytes,
              cudaStream_t st) {
  if (!st) return fail(SFFT_EINVAL, "graph replay needs a non-default stream");
  const void* key[4] = {d_in, d_out, d_scratch, st};
  GraphEntry* gc = nullptr;
  for (GraphEntry& g : cache->e)
    if (g.exec && std::memcmp(key, g.key, sizeof(key)) == 0 && g.bytes == scratch_bytes) gc = &g;
  const bool hit = gc != nullptr;
  if (!hit) {
    gc = cache->e[0].used <= cache->e[1].used ? &cache->e[0] : &cache->e[1];
    if (gc->exec) {
      cudaGraphExecDestroy(gc->exec);
      gc->exec = nullptr;
    }
    // kernel attributes are set outside the capture by a zero-gate launch
    KArgs warm = make_args(s);
    warm.n = 0;
    launch_gates(warm, st);
    cudaGraph_t graph;
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    int rc = ps ? run_persistent(s, dp, *ps, d_in, d_out, d_scratch, scratch_bytes, st, nullptr)
                : run_program(s, dp, d_in, d_out, d_scratch, scratch_bytes, st, nullptr);
    e = cudaStreamEndCapture(st, &graph);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&gc->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    std::memcpy(gc->key, key, sizeof(key));
    gc->bytes = scratch_bytes;
  }
  gc->used = ++cache->clock;
  cudaError_t e = cudaGraphLaunch(gc->exec, st);
  return e == cudaSuccess ? SFFT_OK : cuda_fail(e, "cudaGraphLaunch");
}

}  // namespace sfft

struct sfft_batch {
  sfft::Shape s;
  std::vector<sfft::Program> parts;
  std::vector<std::array<uint64_t, 4>> off;
  sfft::Program merged;
  sfft::DeviceProgram dev;
  sfft::GraphCache graph;
  sfft::Timer timer;
  std::unique_ptr<sfft::PersistState> persist;   // one launch across levels, when requested
  bool use_graph = true;
  uint64_t fft_products = 0;
  // host pipeline: copy streams and the events that order them with the
  // evaluations (created on first use)
  cudaStream_t h2d = nullptr, d2h = nullptr;
  cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_done[2] = {nullptr, nullptr},
              ev_out[2] = {nullptr, nullptr};
  ~sfft_batch() {
    sfft::free_device_program(&dev);
    for (int k = 0; k < 2; k++)
      for (cudaEvent_t ev : {ev_in[k], ev_done[k], ev_out[k]})
        if (ev) cudaEventDestroy(ev);
    if (h2d) cudaStreamDestroy(h2d);
    if (d2h) cudaStreamDestroy(d2h);
  }
};

using namespace sfft;

namespace {

// The persistent form's device state: every gate's level and the gates that
// produced its operands (the last writer of each slot before it, in program
// order), the level widths, and zeroed flags and counters.
int make_persistent(sfft_batch* b) {
  const Program& m = b->merged;
  KArgs k = make_args(b->s);
  k.kernel = b->dev.kernel;
  if (gate_kernel_for(k) != KERNEL_SM)
    return fail(SFFT_EPARAM, "the persistent form runs on the small-ciphertext kernel (64 <= Ng <= 256)");
  const uint32_t levels = (uint32_t)(m.level_off.size() - 1);
  const uint64_t n = m.desc.size();
  if (n >= 0xFFFFFFFFull) return fail(SFFT_EINVAL, "batch too large for the persistent form");
  std::vector<uint32_t> glev, dep_a, dep_b, lwidth;
  if (!persistent_schedule(m, &glev, &dep_a, &dep_b, &lwidth))
    return fail(SFFT_EPARAM, "the persistent form takes circuits without linear gates");
  std::vector<GateDeps> gdep(n);
  for (uint64_t g = 0; g < n; g++) gdep[g] = GateDeps{dep_a[g], dep_b[g]};
  std::unique_ptr<PersistState> ps(new PersistState);
  ps->levels = levels;
  int rc;
  void* p = nullptr;
  if ((rc = upload(glev.data(), n * sizeof(uint32_t), &p))) return rc;
  ps->glev = (uint32_t*)p;
  if ((rc = upload(gdep.data(), n * sizeof(GateDeps), &p))) return rc;
  ps->gdep = (GateDeps*)p;
  if ((rc = upload(lwidth.data(), levels * sizeof(uint32_t), &p))) return rc;
  ps->lwidth = (uint32_t*)p;
  cudaError_t e = cudaMalloc((void**)&ps->ldone, std::max<uint32_t>(levels, 1) * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc((void**)&ps->gflag, std::max<uint64_t>(n, 1) * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&ps->claim, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&ps->epoch, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemset(ps->gflag, 0, std::max<uint64_t>(n, 1) * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemset(ps->epoch, 0, sizeof(uint32_t));
  if (e != cudaSuccess) return cuda_fail(e, "persistent batch state");
  b->persist = std::move(ps);
  return SFFT_OK;
}

}  // namespace

extern "C" {

int sfft_batch_create(const sfft_params* p, const sfft_request* reqs, uint32_t count, uint32_t flags,
                      sfft_batch** out) {
  if (!out || (!reqs && count)) return fail(SFFT_EINVAL, "null argument");
  *out = nullptr;
  if (count == 0) return fail(SFFT_EINVAL, "empty batch");
  std::unique_ptr<sfft_batch> b(new (std::nothrow) sfft_batch);
  if (!b) return fail(SFFT_ENOMEM, "host allocation failed");
  int rc = make_shape(p, &b->s, false);
  if (rc) return rc;
  uint64_t in = 0, outp = 0, scr = 0;
  for (uint32_t r = 0; r < count; r++) {
    Circuit c;
    if (!c.set_variant(flags))
      return fail(SFFT_EINVAL, "SFFT_PLAN_XCARRY and SFFT_PLAN_NAND are exclusive");
    if (!build_fft(&c, reqs[r].N1, reqs[r].N2, reqs[r].F, reqs[r].f))
      return fail(SFFT_EINVAL, "request " + std::to_string(r) + ": invalid FFT shape");
    Program prog;
    // the persistent form overlaps neighbouring levels: slots are reused two
    // levels after their last read
    compile(c, b->s, &prog, 0, (flags & SFFT_BATCH_PERSISTENT) ? 2u : 1u);
    if (!prog.noise_ok && !(flags & SFFT_PLAN_ALLOW_NOISY))
      return fail(SFFT_EPARAM, "request " + std::to_string(r) + ": static noise bound reaches q/4");
    std::array<uint64_t, 4> o = {scr, in, outp, 0};
    b->off.push_back(o);
    scr += prog.scratch_slots;
    in += prog.n_inputs;
    outp += prog.n_outputs;
    b->fft_products += prog.products;
    b->parts.push_back(std::move(prog));
  }
  if (scr > SLOT_MASK || in > SLOT_MASK || outp > SLOT_MASK)
    return fail(SFFT_EINVAL, "batch too large for 30-bit slot numbers");
  merge_programs(b->parts, b->off, &b->merged);
  b->merged.n_inputs = in;
  b->merged.n_outputs = outp;
  b->merged.scratch_slots = scr;
  if ((rc = make_device_program(b->merged, &b->dev))) {
    free_device_program(&b->dev);
    return rc;
  }
  b->dev.kernel = plan_kernel(flags);
  b->dev.max_width = b->merged.max_width;
  {
    KArgs k = make_args(b->s);
    k.kernel = b->dev.kernel;
    if (!gate_kernel_for(k)) return fail(SFFT_EPARAM, "the requested gate kernel does not support these parameters");
    b->dev.tc = gate_kernel_for(k) == KERNEL_TC;   // needs the B expansion region
  }
  b->dev.scratch_bytes =
      scratch_layout(b->s, scr, b->merged.max_width, b->dev.tc, &b->dev.bx_off);
  b->use_graph = !(flags & SFFT_BATCH_NO_GRAPH);
  if ((flags & SFFT_BATCH_PERSISTENT) && (rc = make_persistent(b.get()))) return rc;
  *out = b.release();
  return SFFT_OK;
}

int sfft_batch_info_get(const sfft_batch* b, sfft_plan_info* info) {
  if (!b || !info) return fail(SFFT_EINVAL, "null argument");
  std::memset(info, 0, sizeof(*info));
  info->inputs = b->merged.n_inputs;
  info->outputs = b->merged.n_outputs;
  info->products = b->merged.products;
  info->levels = b->merged.level_off.size() - 1;
  info->max_level_width = b->merged.max_width;
  info->scratch_slots = b->merged.scratch_slots;
  info->scratch_bytes = b->dev.scratch_bytes;
  info->ct_words = b->s.ctw;
  info->noise_bits = b->merged.noise_bits;
  info->noise_ok = b->merged.noise_ok ? 1 : 0;
  KArgs k = make_args(b->s);
  k.kernel = b->dev.kernel;
  info->gate_kernel = gate_kernel_for(k);
  info->tc_columns = gate_digit_columns(k);
  return SFFT_OK;
}

int sfft_batch_offsets(const sfft_batch* b, uint64_t* in_off, uint64_t* out_off) {
  if (!b) return fail(SFFT_EINVAL, "batch is NULL");
  for (size_t r = 0; r < b->off.size(); r++) {
    if (in_off) in_off[r] = b->off[r][REG_IN];
    if (out_off) out_off[r] = b->off[r][REG_OUT];
  }
  return SFFT_OK;
}

int sfft_batch_eval(sfft_batch* b, const uint32_t* d_in, uint32_t* d_out, uint32_t* d_scratch,
                    uint64_t scratch_bytes, void* stream) {
  if (!b) return fail(SFFT_EINVAL, "batch is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  if (b->use_graph && !b->timer.on)
    return run_graph(&b->graph, b->s, b->dev, b->persist.get(), d_in, d_out, d_scratch, scratch_bytes, st);
  if (b->persist)
    return run_persistent(b->s, b->dev, *b->persist, d_in, d_out, d_scratch, scratch_bytes, st, &b->timer);
  return run_program(b->s, b->dev, d_in, d_out, d_scratch, scratch_bytes, st, &b->timer);
}

int sfft_batch_eval_host(sfft_batch* b, const uint32_t* h_in, uint32_t* h_out, uint32_t* d_in,
                         uint32_t* d_out, uint32_t* d_scratch, uint64_t scratch_bytes, void* stream) {
  if (!b || !h_in || !h_out) return fail(SFFT_EINVAL, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  const uint64_t in_b = b->merged.n_inputs * b->s.ctw * 4, out_b = b->merged.n_outputs * b->s.ctw * 4;
  cudaError_t e = cudaMemcpyAsync(d_in, h_in, in_b, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "H2D copy");
  int rc = sfft_batch_eval(b, d_in, d_out, d_scratch, scratch_bytes, stream);
  if (rc) return rc;
  e = cudaMemcpyAsync(h_out, d_out, out_b, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_fail(e, "D2H copy");
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "stream sync");
  return check_device_error(b->dev.err, st);
}

int sfft_batch_eval_host_pipelined(sfft_batch* b, const uint32_t* const* h_in,
                                   uint32_t* const* h_out, uint32_t count,
                                   uint32_t* const* d_in, uint32_t* const* d_out,
                                   uint32_t* d_scratch, uint64_t scratch_bytes, void* stream) {
  if (!b || !h_in || !h_out || !d_in || !d_out) return fail(SFFT_EINVAL, "null argument");
  if (!stream) return fail(SFFT_EINVAL, "the pipeline needs a non-default stream");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (!b->h2d) {
    e = cudaStreamCreateWithFlags(&b->h2d, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->d2h, cudaStreamNonBlocking);
    for (int k = 0; k < 2 && e == cudaSuccess; k++) {
      e = cudaEventCreateWithFlags(&b->ev_in[k], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_done[k], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return cuda_fail(e, "pipeline streams");
  }
  const uint64_t in_b = b->merged.n_inputs * b->s.ctw * 4, out_b = b->merged.n_outputs * b->s.ctw * 4;
  for (uint32_t i = 0; i < count; i++) {
    const uint32_t k = i & 1u;
    if (!h_in[i] || !h_out[i] || !d_in[k] || !d_out[k]) {
      cudaStreamSynchronize(b->h2d);
      cudaStreamSynchronize(b->d2h);
      return fail(SFFT_EINVAL, "null buffer");
    }
    // inputs of step i into set k once step i - 2 has read it
    if (i >= 2 && (e = cudaStreamWaitEvent(b->h2d, b->ev_done[k], 0)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(d_in[k], h_in[i], in_b, cudaMemcpyHostToDevice, b->h2d)) != cudaSuccess)
      break;
    if ((e = cudaEventRecord(b->ev_in[k], b->h2d)) != cudaSuccess) break;
    // evaluation once its inputs landed and step i - 2's outputs left set k
    if ((e = cudaStreamWaitEvent(st, b->ev_in[k], 0)) != cudaSuccess) break;
    if (i >= 2 && (e = cudaStreamWaitEvent(st, b->ev_out[k], 0)) != cudaSuccess) break;
    int rc = sfft_batch_eval(b, d_in[k], d_out[k], d_scratch, scratch_bytes, stream);
    if (rc) {   // leave no copy of this call in flight
      cudaStreamSynchronize(b->h2d);
      cudaStreamSynchronize(b->d2h);
      return rc;
    }
    if ((e = cudaEventRecord(b->ev_done[k], st)) != cudaSuccess) break;
    // outputs back while the next step runs
    if ((e = cudaStreamWaitEvent(b->d2h, b->ev_done[k], 0)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(h_out[i], d_out[k], out_b, cudaMemcpyDeviceToHost, b->d2h)) != cudaSuccess)
      break;
    if ((e = cudaEventRecord(b->ev_out[k], b->d2h)) != cudaSuccess) break;
  }
  cudaError_t s1 = cudaStreamSynchronize(b->h2d), s2 = cudaStreamSynchronize(st),
              s3 = cudaStreamSynchronize(b->d2h);
  if (e != cudaSuccess) return cuda_fail(e, "pipelined evaluation");
  if (s1 != cudaSuccess || s2 != cudaSuccess || s3 != cudaSuccess)
    return cuda_fail(s1 != cudaSuccess ? s1 : s2 != cudaSuccess ? s2 : s3, "stream sync");
  return check_device_error(b->dev.err, st);
}

int sfft_batch_check(sfft_batch* b, void* stream) {
  if (!b) return fail(SFFT_EINVAL, "batch is NULL");
  return check_device_error(b->dev.err, (cudaStream_t)stream);
}

int sfft_batch_set_epoch(sfft_batch* b, uint32_t epoch, void* stream) {
  if (!b) return fail(SFFT_EINVAL, "batch is NULL");
  if (!b->persist) return fail(SFFT_EINVAL, "not a persistent batch");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(b->persist->epoch, &epoch, sizeof(epoch), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? SFFT_OK : cuda_fail(e, "set epoch");
}

int sfft_batch_set_timing(sfft_batch* b, int on) {
  if (!b) return fail(SFFT_EINVAL, "batch is NULL");
  b->timer.drain_ms();
  b->timer.on = on != 0;
  b->timer.launches = b->timer.products = 0;
  return SFFT_OK;
}

int sfft_batch_timing(sfft_batch* b, double* gate_ms, double* expand_ms, uint64_t* launches,
                      uint64_t* products) {
  if (!b) return fail(SFFT_EINVAL, "batch is NULL");
  const double ms = b->timer.drain_ms();
  if (expand_ms) *expand_ms = b->timer.last_expand_ms;
  if (gate_ms) *gate_ms = ms;
  if (launches) *launches = b->timer.launches;
  if (products) *products = b->timer.products;
  b->timer.launches = b->timer.products = 0;
  return SFFT_OK;
}

void sfft_batch_free(sfft_batch* b) {
  if (!b) return;
  free_device_program(&b->dev);
  delete b;
}

}  // extern "C"
