// Host-only C ABI over the circuit compiler: statistics and a plaintext run of
// the compiled device program (same levels, slots, fix-ups and coefficients).
#include <cstring>
#include <vector>

#include "common.h"
#include "kargs.h"
#include "netlist.h"

namespace sfft {
uint64_t tc_bx_bytes(const KArgs& a, uint64_t gates);
uint32_t gate_kernel_for(const KArgs& a);
uint32_t gate_digit_columns(const KArgs& a);
}

using namespace sfft;

namespace {

int nib(uint32_t code, int k) { return (int)((int32_t)(code << (28 - 4 * k)) >> 28); }

int build(const sfft_params* p, const CircuitSpec& spec, uint32_t flags, Shape* s, Circuit* c,
          Program* prog) {
  int rc = make_shape(p, s, false);
  if (rc) return rc;
  if ((rc = build_circuit(c, spec, flags))) return rc;
  compile(*c, *s, prog, level_cap(spec));
  return SFFT_OK;
}

CircuitSpec fft_spec(uint32_t N1, uint32_t N2, uint32_t F, uint32_t f) {
  CircuitSpec sp;
  sp.N1 = N1;
  sp.N2 = N2;
  sp.F = F;
  sp.f = f;
  return sp;
}

CircuitSpec refresh_spec(const sfft_params* p, uint64_t count) {
  CircuitSpec sp;
  sp.op = kOpRefresh;
  sp.count = count;
  sp.n = p ? p->n : 0;
  sp.ell = p ? p->ell : 0;
  return sp;
}

// Bit pos (over the row's n + 1 elements of ell bits) of a public row given
// as (n + 1) L words.
int row_bit(const uint32_t* row, const Shape& s, uint32_t pos) {
  const uint32_t j = pos / s.ell, b = pos % s.ell;
  return (row[j * s.L + b / 32] >> (b % 32)) & 1;
}

uint32_t patched(uint32_t code, int ba, int bb) {
  uint32_t out = 0;
  for (int h = 0; h < 2; h++) {
    const uint32_t k = (code >> (16 * h)) & 0xFFFFu;
    const int c0 = nib(k, 0), c1 = nib(k, 1), c2 = nib(k, 2), c3 = nib(k, 3);
    out |= (uint32_t)pack_code(c0, c1 * ba, c2 * bb, c3 * ba * bb) << (16 * h);
  }
  return out;
}

CircuitSpec word_spec(uint32_t op, uint64_t count, uint32_t F, uint32_t f) {
  CircuitSpec sp;
  sp.op = op;
  sp.count = count;
  sp.F = F;
  sp.f = f;
  return sp;
}


int circuit_info(const sfft_params* p, const CircuitSpec& spec, uint32_t flags,
                 sfft_plan_info* info) {
  if (!info) return fail(SFFT_EINVAL, "info is NULL");
  Shape s;
  Circuit c;
  Program prog;
  int rc = build(p, spec, flags, &s, &c, &prog);
  if (rc) return rc;
  std::memset(info, 0, sizeof(*info));
  info->inputs = prog.n_inputs;
  info->outputs = prog.n_outputs;
  info->gates_and = c.n_and;
  info->gates_xor = c.n_xor;
  info->gates_or = c.n_or;
  info->gates_not = c.n_not;
  info->gates_xadd = c.n_xadd;
  info->products = prog.products;
  info->levels = prog.level_off.size() - 1;
  info->max_level_width = prog.max_width;
  info->scratch_slots = prog.scratch_slots;
  {
    KArgs k{};
    k.Ng = s.Ng;
    k.W = s.W;
    k.L = s.L;
    k.ell = s.ell;
    uint64_t bx_off = 0;
    const bool tc = gate_kernel_for(k) == KERNEL_TC;   // needs the B expansion region
    const uint64_t wires = prog.scratch_slots * s.ctw * 4;
    bx_off = (wires + 255) & ~255ull;
    info->scratch_bytes = tc ? bx_off + tc_bx_bytes(k, prog.max_width) : wires;
  }
  info->ct_words = s.ctw;
  info->noise_bits = prog.noise_bits;
  info->noise_ok = prog.noise_ok ? 1 : 0;
  KArgs ka{};
  ka.Ng = s.Ng;
  ka.W = s.W;
  ka.L = s.L;
  ka.ell = s.ell;
  info->gate_kernel = gate_kernel_for(ka);
  info->tc_columns = gate_digit_columns(ka);
  return SFFT_OK;
}

// h_rows: row ell - 1 of every refreshed ciphertext ((n + 1) L words each),
// for the code patches of a refresh program; NULL otherwise.
int program_eval_plain(const sfft_params* p, const CircuitSpec& spec, uint32_t flags,
                       const uint8_t* h_in_bits, uint8_t* h_out_bits,
                       const uint32_t* h_rows = nullptr) {
  if (!h_in_bits || !h_out_bits) return fail(SFFT_EINVAL, "null argument");
  Shape s;
  Circuit c;
  Program prog;
  int rc = build(p, spec, flags, &s, &c, &prog);
  if (rc) return rc;
  if (!prog.patch.empty() && !h_rows) return fail(SFFT_EINVAL, "refresh rows are NULL");
  for (const PatchDesc& pd : prog.patch) {
    const int ba = pd.a_ct == REF_NONE ? 1 : row_bit(h_rows + (uint64_t)pd.a_ct * s.W, s, pd.a_pos);
    const int bb = pd.b_ct == REF_NONE ? 1 : row_bit(h_rows + (uint64_t)pd.b_ct * s.W, s, pd.b_pos);
    prog.aux[pd.gate].code = patched(pd.code, ba, bb);
  }
  std::vector<int> reg[3];
  reg[REG_SCRATCH].assign(prog.scratch_slots, -1);
  reg[REG_IN].assign(h_in_bits, h_in_bits + prog.n_inputs);
  reg[REG_OUT].assign(prog.n_outputs, -1);
  auto get = [&](uint32_t ref) -> int {
    int v = reg[ref >> 30][ref & SLOT_MASK];
    return v;
  };
  for (size_t g = 0; g < prog.desc.size(); g++) {
    const GateDesc& d = prog.desc[g];
    const GateAux& x = prog.aux[g];
    int a = get(d.a), b = get(d.b);
    if (a < 0 || b < 0) return fail(SFFT_EINVAL, "program reads an unwritten slot");
    int at = (x.flags & 1) ? 1 - a : a;
    uint32_t codes[2] = {x.code & 0xFFFFu, x.code >> 16};
    uint32_t outs[2] = {d.o0, d.o1};
    for (int o = 0; o < 2; o++) {
      if (outs[o] == REF_NONE) continue;
      int v = nib(codes[o], 0) + nib(codes[o], 1) * a + nib(codes[o], 2) * b +
              nib(codes[o], 3) * at * b;
      if (v != 0 && v != 1) return fail(SFFT_EINVAL, "gate produced a non-bit");
      reg[outs[o] >> 30][outs[o] & SLOT_MASK] = v;
    }
  }
  for (const FixDesc& fx : prog.fix) {
    int v;
    if (fx.kind == 2)
      v = 0;
    else if (fx.kind == 3)
      v = 1;
    else {
      v = get(fx.src);
      if (v < 0) return fail(SFFT_EINVAL, "fix-up reads an unwritten slot");
      if (fx.kind == 1) v = 1 - v;
    }
    reg[REG_OUT][fx.dst] = v;
  }
  for (uint64_t o = 0; o < prog.n_outputs; o++) {
    if (reg[REG_OUT][o] < 0) return fail(SFFT_EINVAL, "output never written");
    h_out_bits[o] = (uint8_t)reg[REG_OUT][o];
  }
  return SFFT_OK;
}

}  // namespace

extern "C" {

int sfft_circuit_info(const sfft_params* p, uint32_t N1, uint32_t N2, uint32_t F, uint32_t f,
                      uint32_t flags, sfft_plan_info* info) {
  return circuit_info(p, fft_spec(N1, N2, F, f), flags, info);
}

int sfft_program_eval_plain(const sfft_params* p, uint32_t N1, uint32_t N2, uint32_t F,
                            uint32_t f, uint32_t flags, const uint8_t* h_in_bits, uint8_t* h_out_bits) {
  return program_eval_plain(p, fft_spec(N1, N2, F, f), flags, h_in_bits, h_out_bits);
}

int sfft_word_circuit_info(const sfft_params* p, uint32_t op, uint64_t count, uint32_t F,
                           uint32_t f, uint32_t flags, sfft_plan_info* info) {
  return circuit_info(p, word_spec(op, count, F, f), flags, info);
}

int sfft_word_program_eval_plain(const sfft_params* p, uint32_t op, uint64_t count, uint32_t F,
                                 uint32_t f, uint32_t flags, const uint8_t* h_in_bits,
                                 uint8_t* h_out_bits) {
  return program_eval_plain(p, word_spec(op, count, F, f), flags, h_in_bits, h_out_bits);
}

int sfft_refresh_circuit_info(const sfft_params* p, uint64_t count, uint32_t flags,
                              sfft_plan_info* info) {
  return circuit_info(p, refresh_spec(p, count), flags, info);
}

int sfft_refresh_eval_plain(const sfft_params* p, uint64_t count, uint32_t flags,
                            const uint8_t* h_key_bits, const uint32_t* h_rows,
                            uint8_t* h_out_bits) {
  if (!h_rows) return fail(SFFT_EINVAL, "null argument");
  return program_eval_plain(p, refresh_spec(p, count), flags, h_key_bits, h_out_bits, h_rows);
}

int sfft_program_gates(const sfft_params* p, uint32_t N1, uint32_t N2, uint32_t F, uint32_t f,
                       uint32_t flags, sfft_gate_record* h_gates, uint64_t capacity, uint64_t* count) {
  if (!count) return fail(SFFT_EINVAL, "count is NULL");
  const CircuitSpec spec = fft_spec(N1, N2, F, f);
  Shape s;
  Circuit c;
  Program prog;
  int rc = make_shape(p, &s, false);
  if (rc) return rc;
  if ((rc = build_circuit(&c, spec, flags))) return rc;
  const bool persist = (flags & SFFT_BATCH_PERSISTENT) != 0;
  compile(c, s, &prog, level_cap(spec), persist ? 2u : 1u);
  const uint64_t n = prog.desc.size();
  *count = n;
  if (!h_gates) return SFFT_OK;
  if (capacity < n) return fail(SFFT_EINVAL, "capacity below the gate count");
  std::vector<uint32_t> glev, dep_a, dep_b, lwidth;
  if (persist && !persistent_schedule(prog, &glev, &dep_a, &dep_b, &lwidth))
    return fail(SFFT_EPARAM, "the persistent form takes circuits without linear gates");
  const uint32_t levels = (uint32_t)(prog.level_off.size() - 1);
  for (uint32_t l = 0; l < levels; l++)
    for (uint64_t g = prog.level_off[l]; g < prog.level_off[l + 1]; g++) {
      sfft_gate_record& r = h_gates[g];
      r.a = prog.desc[g].a;
      r.b = prog.desc[g].b;
      r.o0 = prog.desc[g].o0;
      r.o1 = prog.desc[g].o1;
      r.code = prog.aux[g].code;
      r.flags = prog.aux[g].flags;
      r.level = l;
      r.dep_a = persist ? dep_a[g] : 0xFFFFFFFFu;
      r.dep_b = persist ? dep_b[g] : 0xFFFFFFFFu;
    }
  return SFFT_OK;
}

int sfft_twiddles(uint32_t M, uint32_t f, int64_t* h_wr, int64_t* h_wi) {
  if (M < 2 || (M & (M - 1)) || f > 62) return fail(SFFT_EINVAL, "M must be a power of two >= 2, f <= 62");
  if (!h_wr || !h_wi) return fail(SFFT_EINVAL, "null argument");
  std::vector<int64_t> wr, wi;
  twiddles(M, f, &wr, &wi);
  std::memcpy(h_wr, wr.data(), wr.size() * sizeof(int64_t));
  std::memcpy(h_wi, wi.data(), wi.size() * sizeof(int64_t));
  return SFFT_OK;
}

}  // extern "C"
