// C ABI: FFT plans and the plain level-by-level evaluator, device encryption,
// the single-level gate hook and decryption-row gathering.
#include <cuda_runtime.h>

#include <atomic>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "common.h"
#include "kernels.cuh"
#include "netlist.h"
#include "plan.h"
#include "scheme.h"

namespace sfft {

int cuda_fail(cudaError_t e, const char* what) {
  return fail(SFFT_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int upload(const void* h, size_t bytes, void** d) {
  *d = nullptr;
  if (bytes == 0) return SFFT_OK;
  cudaError_t e = cudaMalloc(d, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  e = cudaMemcpy(*d, h, bytes, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
  return SFFT_OK;
}

KArgs make_args(const Shape& s) {
  KArgs a{};
  a.Ng = s.Ng;
  a.W = s.W;
  a.L = s.L;
  a.ell = s.ell;
  a.ctw = s.ctw;
  return a;
}

static std::atomic<uint64_t> g_launches{0};
void count_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

uint64_t scratch_layout(const Shape& s, uint64_t slots, uint64_t max_width, bool tc, uint64_t* bx_off) {
  const uint64_t wires = slots * s.ctw * 4;
  *bx_off = (wires + 255) & ~255ull;
  if (!tc) return wires;
  return *bx_off + tc_bx_bytes(make_args(s), max_width);
}

uint32_t gate_kernel_for(const KArgs& a) {
  switch (a.kernel) {
    case KERNEL_INT:
      return KERNEL_INT;
    case KERNEL_TC:
      return tc_supported(a) ? KERNEL_TC : 0;
    case KERNEL_SM:
      return !a.bx_shared && !a.gen_state && sm_supported(a) ? KERNEL_SM : 0;
    default:
      // the small-ciphertext kernel where it applies (it loads both operands
      // of each gate; encryption, whose A operands are generated and whose
      // gates share one expanded B, runs the general one)
      if (!a.bx_shared && !a.gen_state && sm_supported(a)) return KERNEL_SM;
      return tc_supported(a) ? KERNEL_TC : KERNEL_INT;
  }
}

uint32_t plan_kernel(uint32_t flags) {
  if (flags & SFFT_PLAN_INT_KERNEL) return KERNEL_INT;
  if (flags & SFFT_PLAN_TC_KERNEL) return KERNEL_TC;
  return KERNEL_AUTO;
}

uint32_t gate_digit_columns(const KArgs& a) {
  const uint32_t k = gate_kernel_for(a);
  return k == KERNEL_SM ? sm_digit_columns(a) : k == KERNEL_TC ? tc_digit_columns(a) : 0;
}

// Launches one level of gates on the kernel gate_kernel_for picks.
int launch_gates(const KArgs& a, cudaStream_t st) {
  if (a.n == 0) return SFFT_OK;
  const uint32_t k = gate_kernel_for(a);
  if (k == KERNEL_SM) return launch_gates_sm(a, st);
  if (k == KERNEL_TC) return launch_gates_tc(a, st);
  if (k == 0) return fail(SFFT_EPARAM, "the requested gate kernel does not support this shape");
  const uint64_t tasks = a.n * (a.Ng / 32);
  const uint64_t blocks = (tasks * 32 + 255) / 256;
  Timer* tm = static_cast<Timer*>(a.timer);
  if (tm) cudaEventRecord(tm->next(kTimeGate), st);
  if (a.W <= 2)
    k_gate_generic<2><<<(unsigned)blocks, 256, 0, st>>>(a);
  else if (a.W <= 4)
    k_gate_generic<4><<<(unsigned)blocks, 256, 0, st>>>(a);
  else
    k_gate_generic<8><<<(unsigned)blocks, 256, 0, st>>>(a);
  if (tm) cudaEventRecord(tm->next(kTimeGate), st);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SFFT_OK : cuda_fail(e, "gate kernel launch");
}

cudaEvent_t Timer::next(int kind) {
  if (used[kind] == pool[kind].size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    pool[kind].push_back(e);
  }
  return pool[kind][used[kind]++];
}

double Timer::drain_ms() {
  double ms[2] = {0, 0};
  for (int kind = 0; kind < 2; kind++) {
    for (size_t k = 0; k + 1 < used[kind]; k += 2) {
      cudaEventSynchronize(pool[kind][k + 1]);
      float t = 0;
      cudaEventElapsedTime(&t, pool[kind][k], pool[kind][k + 1]);
      ms[kind] += t;
    }
    used[kind] = 0;
  }
  last_expand_ms = ms[kTimeExpand];
  return ms[kTimeGate];
}

Timer::~Timer() {
  for (auto& p : pool)
    for (cudaEvent_t e : p) cudaEventDestroy(e);
}

int run_program(const Shape& s, const DeviceProgram& dp, const uint32_t* d_in, uint32_t* d_out,
                uint32_t* d_scratch, uint64_t scratch_bytes, cudaStream_t st, Timer* tm) {
  const uint32_t levels = (uint32_t)(dp.level_off.size() - 1);
  return run_levels(s, dp, 0, levels, d_in, d_out, d_scratch, scratch_bytes, st, tm);
}

int run_levels(const Shape& s, const DeviceProgram& dp, uint32_t l0, uint32_t l1, const uint32_t* d_in,
               uint32_t* d_out, uint32_t* d_scratch, uint64_t scratch_bytes, cudaStream_t st, Timer* tm) {
  if (!d_in || !d_out) return fail(SFFT_EINVAL, "null buffer");
  const uint32_t levels = (uint32_t)(dp.level_off.size() - 1);
  if (l0 > l1 || l1 > levels) return fail(SFFT_EINVAL, "level range out of bounds");
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != dp.device)
    return fail(SFFT_EINVAL, "the current CUDA device is not the one the plan was created on");
  if (scratch_bytes < dp.scratch_bytes || (dp.scratch_bytes && !d_scratch))
    return fail(SFFT_EINVAL, "scratch buffer too small");
  KArgs a = make_args(s);
  a.base[REG_SCRATCH] = d_scratch;
  a.bx = dp.tc ? (uint8_t*)d_scratch + dp.bx_off : nullptr;
  a.base[REG_IN] = const_cast<uint32_t*>(d_in);
  a.base[REG_OUT] = d_out;
  a.base[REG_GEN] = nullptr;
  a.err = dp.err;
  a.kernel = dp.kernel;
  for (size_t l = l0; l < l1; l++) {
    const uint64_t mid = dp.lin_start[l];
    a.desc = dp.desc + dp.level_off[l];
    a.aux = dp.aux + dp.level_off[l];
    a.n = mid - dp.level_off[l];
    const bool timed = tm && tm->on && a.n;
    a.timer = timed ? tm : nullptr;   // the gate launchers record their kernels
    int rc = launch_gates(a, st);
    a.timer = nullptr;
    if (rc) return rc;
    if (timed) {
      tm->launches++;
      tm->products += a.n;
    }
    a.desc = dp.desc + mid;
    a.aux = dp.aux + mid;
    a.n = dp.level_off[l + 1] - mid;
    if ((rc = launch_linear(a, st))) return rc;
  }
  return l1 == levels ? launch_fixups(dp.fix, dp.n_fix, a, st) : SFFT_OK;
}

int launch_linear(const KArgs& a, cudaStream_t st) {
  if (a.n == 0) return SFFT_OK;
  const uint32_t tasks = a.Ng * (a.W / a.L), per = (tasks + 255) / 256;
  k_linear<<<(unsigned)(a.n * per), 256, 0, st>>>(a, per);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SFFT_OK : cuda_fail(e, "linear gate launch");
}

int launch_fixups(const FixDesc* d_fix, uint64_t n, const KArgs& a, cudaStream_t st) {
  if (n == 0) return SFFT_OK;
  k_fixup<<<(unsigned)n, 256, 0, st>>>(d_fix, n, a);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SFFT_OK : cuda_fail(e, "fixup launch");
}

int make_device_program(const Program& p, DeviceProgram* dp) {
  int rc;
  void* ptr;
  if ((rc = upload(p.desc.data(), p.desc.size() * sizeof(GateDesc), &ptr))) return rc;
  dp->desc = (GateDesc*)ptr;
  if ((rc = upload(p.aux.data(), p.aux.size() * sizeof(GateAux), &ptr))) return rc;
  dp->aux = (GateAux*)ptr;
  if ((rc = upload(p.fix.data(), p.fix.size() * sizeof(FixDesc), &ptr))) return rc;
  dp->fix = (FixDesc*)ptr;
  dp->n_fix = p.fix.size();
  if (!p.patch.empty()) {
    if ((rc = upload(p.patch.data(), p.patch.size() * sizeof(PatchDesc), &ptr))) return rc;
    dp->patch = (PatchDesc*)ptr;
    dp->n_patch = p.patch.size();
  }
  if (cudaGetDevice(&dp->device) != cudaSuccess) dp->device = -1;
  dp->level_off = p.level_off;
  dp->lin_start = p.lin_start;
  dp->scratch_slots = p.scratch_slots;
  cudaError_t e = cudaMalloc((void**)&dp->err, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  e = cudaMemset(dp->err, 0, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemset");
  return SFFT_OK;
}

int check_device_error(int* err, cudaStream_t st) {
  if (!err) return SFFT_OK;
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "reading the device error word");
  if (h == 0) return SFFT_OK;
  cudaMemsetAsync(err, 0, sizeof(int), st);
  return fail(SFFT_ETIMEOUT, "a bounded wait inside the tensor-core gate kernel ran out");
}

void free_device_program(DeviceProgram* dp) {
  cudaFree(dp->desc);
  cudaFree(dp->aux);
  cudaFree(dp->fix);
  cudaFree(dp->patch);
  cudaFree(dp->err);
  dp->patch = nullptr;
  dp->n_patch = 0;
  dp->err = nullptr;
  dp->desc = nullptr;
  dp->aux = nullptr;
  dp->fix = nullptr;
}

}  // namespace sfft

using namespace sfft;

namespace {

// One level of independent gates (test hooks): operand A in d_a, B in d_b.
int gate_level(const sfft_params* p, const uint32_t* d_a, const uint32_t* d_b, uint32_t* d_out0,
               uint32_t* d_out1, const uint16_t* h_code0, const uint16_t* h_code1,
               const uint8_t* h_flags, uint64_t n_gates, uint32_t kernel, uint32_t withhold,
               void* stream);

}  // namespace

namespace {

uint32_t min_ell_of(const CircuitSpec& spec, uint32_t n, uint32_t chi, uint32_t flags) {
  Circuit c;
  if (build_circuit(&c, spec, flags)) return 0;
  for (uint32_t ell = 32; ell <= 8192; ell += 32) {
    sfft_params p{n, ell, (n + 1) * ell, chi};
    Shape s;
    if (make_shape(&p, &s, false)) return 0;
    if (noise_bits(c, s) <= ell - 2) return ell;
  }
  return 0;
}

int plan_create(const sfft_params* p, const CircuitSpec& spec, uint32_t flags, sfft_plan** out) {
  if (!out) return fail(SFFT_EINVAL, "out is NULL");
  *out = nullptr;
  std::unique_ptr<sfft_plan> pl(new (std::nothrow) sfft_plan);
  if (!pl) return fail(SFFT_ENOMEM, "host allocation failed");
  int rc = make_shape(p, &pl->s, false);
  if (rc) return rc;
  if ((rc = build_circuit(&pl->circuit, spec, flags))) return rc;
  compile(pl->circuit, pl->s, &pl->prog, level_cap(spec));
  if (spec.op == kOpRefresh) {   // refreshed outputs must be refreshable again
    if (pl->prog.noise_bits > pl->s.ell - 3 && !(flags & SFFT_PLAN_ALLOW_NOISY))
      return fail(SFFT_EPARAM, "refresh output bound reaches q/8: raise ell "
                               "(see sfft_refresh_min_ell)");
  } else if (!pl->prog.noise_ok && !(flags & SFFT_PLAN_ALLOW_NOISY)) {
    return fail(SFFT_EPARAM, "static noise bound reaches q/4: raise ell (see sfft_min_ell)");
  }
  if ((rc = make_device_program(pl->prog, &pl->dev))) {
    free_device_program(&pl->dev);
    return rc;
  }
  pl->spec = spec;
  pl->dev.kernel = plan_kernel(flags);
  pl->dev.max_width = pl->prog.max_width;
  {
    KArgs k = make_args(pl->s);
    k.kernel = pl->dev.kernel;
    if (!gate_kernel_for(k)) return fail(SFFT_EPARAM, "the requested gate kernel does not support these parameters");
    pl->dev.tc = gate_kernel_for(k) == KERNEL_TC;   // needs the B expansion region
  }
  pl->dev.scratch_bytes = scratch_layout(pl->s, pl->prog.scratch_slots, pl->prog.max_width,
                                         pl->dev.tc, &pl->dev.bx_off);
  *out = pl.release();
  return SFFT_OK;
}

}  // namespace

extern "C" {

const char* sfft_version(void) { return "sfft-gb300 0.1 (sm_103a)"; }

uint64_t sfft_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

uint32_t sfft_min_ell(uint32_t N1, uint32_t N2, uint32_t F, uint32_t f, uint32_t n, uint32_t chi,
                      uint32_t flags) {
  CircuitSpec spec;
  spec.N1 = N1;
  spec.N2 = N2;
  spec.F = F;
  spec.f = f;
  return min_ell_of(spec, n, chi, flags);
}

uint32_t sfft_word_min_ell(uint32_t op, uint32_t F, uint32_t f, uint32_t n, uint32_t chi,
                           uint32_t flags) {
  CircuitSpec spec;
  spec.op = op;
  spec.count = 1;
  spec.F = F;
  spec.f = f;
  return min_ell_of(spec, n, chi, flags);
}

int sfft_plan_create(const sfft_params* p, uint32_t N1, uint32_t N2, uint32_t F, uint32_t f,
                     uint32_t flags, sfft_plan** out) {
  CircuitSpec spec;
  spec.N1 = N1;
  spec.N2 = N2;
  spec.F = F;
  spec.f = f;
  return plan_create(p, spec, flags, out);
}

int sfft_word_plan_create(const sfft_params* p, uint32_t op, uint64_t count, uint32_t F,
                          uint32_t f, uint32_t flags, sfft_plan** out) {
  CircuitSpec spec;
  spec.op = op;
  spec.count = count;
  spec.F = F;
  spec.f = f;
  return plan_create(p, spec, flags, out);
}

int sfft_plan_info_get(const sfft_plan* pl, sfft_plan_info* info) {
  if (!pl || !info) return fail(SFFT_EINVAL, "null argument");
  std::memset(info, 0, sizeof(*info));
  info->inputs = pl->prog.n_inputs;
  info->outputs = pl->prog.n_outputs;
  info->gates_and = pl->circuit.n_and;
  info->gates_xor = pl->circuit.n_xor;
  info->gates_or = pl->circuit.n_or;
  info->gates_not = pl->circuit.n_not;
  info->gates_xadd = pl->circuit.n_xadd;
  info->products = pl->prog.products;
  info->levels = pl->prog.level_off.size() - 1;
  info->max_level_width = pl->prog.max_width;
  info->scratch_slots = pl->prog.scratch_slots;
  info->scratch_bytes = pl->dev.scratch_bytes;
  info->ct_words = pl->s.ctw;
  info->noise_bits = pl->prog.noise_bits;
  info->noise_ok = pl->prog.noise_ok ? 1 : 0;
  KArgs k = make_args(pl->s);
  k.kernel = pl->dev.kernel;
  info->gate_kernel = gate_kernel_for(k);
  info->tc_columns = gate_digit_columns(k);
  return SFFT_OK;
}

void sfft_plan_free(sfft_plan* pl) {
  if (!pl) return;
  free_device_program(&pl->dev);
  delete pl;
}

int sfft_eval_fft(sfft_plan* pl, const uint32_t* d_in, uint32_t* d_out, uint32_t* d_scratch,
                  uint64_t scratch_bytes, void* stream) {
  if (!pl) return fail(SFFT_EINVAL, "plan is NULL");
  if (pl->dev.n_patch) return fail(SFFT_EINVAL, "a refresh plan runs through sfft_refresh");
  return run_program(pl->s, pl->dev, d_in, d_out, d_scratch, scratch_bytes, (cudaStream_t)stream,
                     &pl->timer);
}

int sfft_refresh_plan_create(const sfft_params* p, uint64_t count, uint32_t flags,
                             sfft_plan** out) {
  CircuitSpec spec;
  spec.op = kOpRefresh;
  spec.count = count;
  spec.n = p ? p->n : 0;
  spec.ell = p ? p->ell : 0;
  return plan_create(p, spec, flags, out);
}

uint32_t sfft_refresh_min_ell(uint32_t n, uint32_t chi, uint32_t flags) {
  for (uint32_t ell = 32; ell <= 8192; ell += 32) {
    sfft_params p{n, ell, (n + 1) * ell, chi};
    Shape s;
    if (make_shape(&p, &s, false)) return 0;
    CircuitSpec spec;
    spec.op = kOpRefresh;
    spec.count = 1;
    spec.n = n;
    spec.ell = ell;
    Circuit c;
    if (build_circuit(&c, spec, flags)) {
      set_error("");
      continue;   // ell too small for the p-bit sum
    }
    if (noise_bits(c, s) <= ell - 3) return ell;
  }
  return 0;
}

int sfft_refresh(sfft_plan* pl, const uint32_t* d_bk, const uint32_t* d_src, uint32_t* d_out,
                 uint32_t* d_scratch, uint64_t scratch_bytes, void* stream) {
  if (!pl || !d_src) return fail(SFFT_EINVAL, "null argument");
  if (pl->spec.op != kOpRefresh) return fail(SFFT_EINVAL, "not a refresh plan");
  cudaStream_t st = (cudaStream_t)stream;
  const uint64_t n = pl->dev.n_patch;
  if (n) {
    k_patch_codes<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        pl->dev.patch, n, pl->dev.aux, d_src, pl->s.ctw, (pl->s.ell - 1) * pl->s.W, pl->s.L,
        pl->s.ell);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "code patch launch");
  }
  return run_program(pl->s, pl->dev, d_bk, d_out, d_scratch, scratch_bytes, st, &pl->timer);
}

int sfft_plan_set_timing(sfft_plan* pl, int on) {
  if (!pl) return fail(SFFT_EINVAL, "plan is NULL");
  pl->timer.drain_ms();
  pl->timer.on = on != 0;
  pl->timer.launches = pl->timer.products = 0;
  return SFFT_OK;
}

int sfft_plan_timing(sfft_plan* pl, double* gate_ms, double* expand_ms, uint64_t* launches,
                     uint64_t* products) {
  if (!pl) return fail(SFFT_EINVAL, "plan is NULL");
  double ms = pl->timer.drain_ms();
  if (gate_ms) *gate_ms = ms;
  if (expand_ms) *expand_ms = pl->timer.last_expand_ms;
  if (launches) *launches = pl->timer.launches;
  if (products) *products = pl->timer.products;
  pl->timer.launches = pl->timer.products = 0;
  return SFFT_OK;
}

int sfft_eval_fft_host(sfft_plan* pl, const uint32_t* h_in, uint32_t* h_out, uint32_t* d_in,
                       uint32_t* d_out, uint32_t* d_scratch, uint64_t scratch_bytes,
                       void* stream) {
  if (!pl || !h_in || !h_out) return fail(SFFT_EINVAL, "null argument");
  if (pl->dev.n_patch) return fail(SFFT_EINVAL, "a refresh plan runs through sfft_refresh");
  cudaStream_t st = (cudaStream_t)stream;
  const uint64_t in_b = pl->prog.n_inputs * pl->s.ctw * 4, out_b = pl->prog.n_outputs * pl->s.ctw * 4;
  cudaError_t e = cudaMemcpyAsync(d_in, h_in, in_b, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "H2D copy");
  int rc = run_program(pl->s, pl->dev, d_in, d_out, d_scratch, scratch_bytes, st, &pl->timer);
  if (rc) return rc;
  e = cudaMemcpyAsync(h_out, d_out, out_b, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_fail(e, "D2H copy");
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "stream sync");
  return check_device_error(pl->dev.err, st);
}

int sfft_plan_check(sfft_plan* pl, void* stream) {
  if (!pl) return fail(SFFT_EINVAL, "plan is NULL");
  return check_device_error(pl->dev.err, (cudaStream_t)stream);
}

int sfft_eval_levels(sfft_plan* pl, uint32_t l0, uint32_t l1, const uint32_t* d_in, uint32_t* d_out,
                     uint32_t* d_scratch, uint64_t scratch_bytes, void* stream) {
  if (!pl) return fail(SFFT_EINVAL, "plan is NULL");
  if (pl->dev.n_patch) return fail(SFFT_EINVAL, "a refresh plan runs through sfft_refresh");
  return run_levels(pl->s, pl->dev, l0, l1, d_in, d_out, d_scratch, scratch_bytes, (cudaStream_t)stream,
                    nullptr);
}

int sfft_plan_level(const sfft_plan* pl, uint32_t level, uint32_t* h_desc, uint32_t* h_code,
                    uint8_t* h_flags, uint64_t cap, uint64_t* n_gates, uint64_t* n_products) {
  if (!pl || !n_gates) return fail(SFFT_EINVAL, "null argument");
  const Program& p = pl->prog;
  if (level + 1 >= p.level_off.size()) return fail(SFFT_EINVAL, "level out of range");
  const uint64_t g0 = p.level_off[level], g1 = p.level_off[level + 1];
  *n_gates = g1 - g0;
  if (n_products) *n_products = p.lin_start[level] - g0;
  if (!h_desc && !h_code && !h_flags) return SFFT_OK;
  if (cap < g1 - g0) return fail(SFFT_EINVAL, "arrays too small for the level");
  for (uint64_t g = g0; g < g1; g++) {
    const GateDesc& d = p.desc[g];
    if (h_desc) {
      h_desc[4 * (g - g0)] = d.a;
      h_desc[4 * (g - g0) + 1] = d.b;
      h_desc[4 * (g - g0) + 2] = d.o0;
      h_desc[4 * (g - g0) + 3] = d.o1;
    }
    if (h_code) h_code[g - g0] = p.aux[g].code;
    if (h_flags) h_flags[g - g0] = (uint8_t)(p.aux[g].flags & 0xFFu);
  }
  return SFFT_OK;
}

int sfft_gate_level(const sfft_params* p, const uint32_t* d_a, const uint32_t* d_b,
                    uint32_t* d_out0, uint32_t* d_out1, const uint16_t* h_code0,
                    const uint16_t* h_code1, const uint8_t* h_flags, uint64_t n_gates,
                    uint32_t kernel, void* stream) {
  return gate_level(p, d_a, d_b, d_out0, d_out1, h_code0, h_code1, h_flags, n_gates, kernel, 0,
                    stream);
}

int sfft_gate_level_withheld(const sfft_params* p, const uint32_t* d_a, const uint32_t* d_b,
                             uint32_t* d_out0, const uint16_t* h_code0, const uint8_t* h_flags,
                             uint64_t n_gates, uint32_t step, void* stream) {
  Shape s;
  KArgs probe{};
  if (make_shape(p, &s, false) == SFFT_OK) probe = make_args(s);
  if (!tc_supported(probe)) return fail(SFFT_EPARAM, "the tensor-core kernel does not take these parameters");
  return gate_level(p, d_a, d_b, d_out0, nullptr, h_code0, nullptr, h_flags, n_gates, KERNEL_TC,
                    step + 1, stream);
}

}  // extern "C"

namespace {

int gate_level(const sfft_params* p, const uint32_t* d_a, const uint32_t* d_b, uint32_t* d_out0,
               uint32_t* d_out1, const uint16_t* h_code0, const uint16_t* h_code1,
               const uint8_t* h_flags, uint64_t n_gates, uint32_t kernel, uint32_t withhold,
               void* stream) {
  Shape s;
  int rc = make_shape(p, &s, false);
  if (rc) return rc;
  if (!d_a || !d_b || !d_out0 || !h_code0 || !h_flags) return fail(SFFT_EINVAL, "null argument");
  if (n_gates == 0) return SFFT_OK;
  std::vector<GateDesc> desc(n_gates);
  std::vector<GateAux> aux(n_gates);
  for (uint64_t g = 0; g < n_gates; g++) {
    const bool two = (h_flags[g] & 2) && d_out1;
    desc[g] = GateDesc{make_ref(REG_SCRATCH, (uint32_t)g), make_ref(REG_IN, (uint32_t)g),
                       make_ref(REG_OUT, (uint32_t)g), two ? make_ref(REG_GEN, (uint32_t)g) : REF_NONE};
    aux[g].code = (uint32_t)h_code0[g] | ((uint32_t)(two ? h_code1[g] : 0) << 16);
    aux[g].flags = h_flags[g] & 1u;
  }
  cudaStream_t st = (cudaStream_t)stream;
  void *dd = nullptr, *da = nullptr;
  if ((rc = upload(desc.data(), desc.size() * sizeof(GateDesc), &dd))) return rc;
  if ((rc = upload(aux.data(), aux.size() * sizeof(GateAux), &da))) {
    cudaFree(dd);
    return rc;
  }
  KArgs a = make_args(s);
  a.desc = (const GateDesc*)dd;
  a.aux = (const GateAux*)da;
  a.n = n_gates;
  a.base[REG_SCRATCH] = const_cast<uint32_t*>(d_a);
  a.base[REG_IN] = const_cast<uint32_t*>(d_b);
  a.base[REG_OUT] = d_out0;
  a.base[REG_GEN] = d_out1;  // region 3 is only an output here, never operand A
  a.kernel = kernel;
  cudaMalloc((void**)&a.err, sizeof(int));
  if (a.err) cudaMemset(a.err, 0, sizeof(int));
  if (gate_kernel_for(a) == KERNEL_TC) {
    cudaError_t me = cudaMalloc((void**)&a.bx, tc_bx_bytes(a, n_gates));
    if (me != cudaSuccess) {
      cudaFree(dd);
      cudaFree(da);
      cudaFree(a.err);
      return cuda_fail(me, "cudaMalloc");
    }
  }
  rc = withhold ? launch_gates_tc_withheld(a, withhold - 1, st) : launch_gates(a, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (!rc && e == cudaSuccess) rc = check_device_error(a.err, st);
  cudaFree(dd);
  cudaFree(da);
  cudaFree(a.err);
  cudaFree(a.bx);
  if (rc) return rc;
  return e == cudaSuccess ? SFFT_OK : cuda_fail(e, "gate level");
}

}  // namespace

extern "C" {

int sfft_encrypt_bits_device(const sfft_params* p, const uint32_t* d_pub, const double* h_re,
                             const double* h_im, uint64_t count, uint32_t F, uint32_t f,
                             uint64_t enc_seed, uint32_t* d_ct_out, void* stream) {
  if (!h_re) return fail(SFFT_EINVAL, "null argument");
  if (F < 2 || F > 48 || f >= F) return fail(SFFT_EPARAM, "need 2 <= F <= 48 and f < F");
  std::vector<uint8_t> bits;
  encode_signal(h_re, h_im, count, F, f, &bits);
  return sfft_encrypt_raw_bits_device(p, d_pub, bits.data(), bits.size(), enc_seed, d_ct_out,
                                      stream);
}

int sfft_encrypt_raw_bits_device(const sfft_params* p, const uint32_t* d_pub,
                                 const uint8_t* h_bits, uint64_t count, uint64_t enc_seed,
                                 uint32_t* d_ct_out, void* stream) {
  Shape s;
  int rc = make_shape(p, &s, true);
  if (rc) return rc;
  if (!d_pub || !h_bits || !d_ct_out) return fail(SFFT_EINVAL, "null argument");
  if (count == 0) return SFFT_OK;
  std::vector<uint8_t> bits(h_bits, h_bits + count);
  for (uint8_t& b : bits)
    if (b > 1) return fail(SFFT_EINVAL, "bits must be 0 or 1");
  const uint64_t n = bits.size();
  std::vector<GateDesc> desc(n);
  std::vector<GateAux> aux(n);
  for (uint64_t c = 0; c < n; c++) {
    desc[c] = GateDesc{make_ref(REG_GEN, (uint32_t)c), make_ref(REG_IN, 0),
                       make_ref(REG_OUT, (uint32_t)c), REF_NONE};
    aux[c].code = pack_code(bits[c], 0, 0, 1);   // mu P + BitDecomp(R) A
    aux[c].flags = 0;
  }
  void *dd = nullptr, *da = nullptr;
  if ((rc = upload(desc.data(), n * sizeof(GateDesc), &dd))) return rc;
  if ((rc = upload(aux.data(), n * sizeof(GateAux), &da))) {
    cudaFree(dd);
    return rc;
  }
  KArgs a = make_args(s);
  a.desc = (const GateDesc*)dd;
  a.aux = (const GateAux*)da;
  a.n = n;
  a.base[REG_IN] = const_cast<uint32_t*>(d_pub);
  a.base[REG_OUT] = d_ct_out;
  a.gen_state = domain_key(enc_seed, kDomR);
  cudaStream_t st = (cudaStream_t)stream;
  if (tc_supported(a)) {  // every gate multiplies by the same public matrix: expand it once
    a.bx_shared = 1;
    cudaError_t me = cudaMalloc((void**)&a.bx, tc_bx_bytes_per_gate(a));
    if (me != cudaSuccess) {
      cudaFree(dd);
      cudaFree(da);
      return cuda_fail(me, "cudaMalloc");
    }
  }
  rc = launch_gates(a, st);
  cudaError_t e = cudaStreamSynchronize(st);
  cudaFree(dd);
  cudaFree(da);
  cudaFree(a.bx);
  if (rc) return rc;
  return e == cudaSuccess ? SFFT_OK : cuda_fail(e, "device encryption");
}

int sfft_gather_dec_rows(const sfft_params* p, const uint32_t* d_ct, uint64_t n_ct,
                         uint32_t* d_rows, void* stream) {
  Shape s;
  int rc = make_shape(p, &s, false);
  if (rc) return rc;
  if (!d_ct || !d_rows) return fail(SFFT_EINVAL, "null argument");
  if (n_ct == 0) return SFFT_OK;
  const uint64_t t = n_ct * s.W;
  k_gather_rows<<<(unsigned)((t + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      d_ct, n_ct, s.ctw, s.W, s.ell - 1, d_rows);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SFFT_OK : cuda_fail(e, "gather rows");
}

}  // extern "C"
