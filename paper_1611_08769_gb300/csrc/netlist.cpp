// Canonical FFT gate circuit, levelisation, slot allocation, noise bound.
#include "netlist.h"

#include <algorithm>
#include <cmath>

namespace sfft {

// ------------------------------------------------------------------ circuit

bool Circuit::set_variant(uint32_t flags) {
  xcarry = (flags & SFFT_PLAN_XCARRY) != 0;
  nand = (flags & SFFT_PLAN_NAND) != 0;
  enc_twiddle = (flags & SFFT_PLAN_ENC_TWIDDLE) != 0;
  return !(xcarry && nand);
}

uint32_t Circuit::new_node(uint32_t d, int32_t prod) {
  if (depth.empty()) {  // node 0: the constant zero
    depth.push_back(0);
    producer.push_back(-1);
  }
  depth.push_back(d);
  producer.push_back(prod);
  return (uint32_t)depth.size() - 1;
}

uint32_t Circuit::new_input() {
  uint32_t n = new_node(0, -1);
  inputs.push_back(n);
  return n;
}

Sig Circuit::NOT(Sig a) {
  if (sig_node(a) != 0) n_not++;
  if (nand && sig_node(a) != 0) return NAND(a, a);
  return a ^ SIG_ONE;
}

Sig Circuit::SEL(uint32_t input, uint32_t src_ct, uint32_t src_pos) {
  const uint32_t node = new_node(0, -1);
  vin_of[node] = (uint32_t)vin.size();
  vin.push_back(VInput{input, src_ct, src_pos});
  return node;
}

Sig Circuit::AND(Sig a, Sig b) {
  if (a == SIG_ZERO || b == SIG_ZERO) return SIG_ZERO;
  if (a == SIG_ONE) return b;
  if (b == SIG_ONE) return a;
  if (nand) {
    n_and++;
    const Sig t = NAND(a, b);
    return NOT(t);
  }
  Sig s, c;
  const uint64_t xors = n_xor;
  HA(a, b, &s, &c);   // the XOR output stays unused (pruned)
  n_xor = xors;
  return c;
}

Sig Circuit::NAND(Sig a, Sig b) {
  uint32_t d = 1 + std::max(dep(a), dep(b));
  Product p;
  if (dep(b) > dep(a)) {
    p.a = b;
    p.b = a;
  } else {
    p.a = a;
    p.b = b;
  }
  p.is_or = false;
  p.is_add = false;
  p.is_nand = true;
  p.out_and = 0;
  const uint64_t key = ((uint64_t)p.a << 32) | p.b;
  auto hit = memo_nand.find(key);
  if (hit != memo_nand.end()) return products[hit->second].out_xor;
  int32_t id = (int32_t)products.size();
  memo_nand[key] = id;
  products.push_back(p);
  uint32_t n = new_node(d, id);
  products[id].out_xor = n;
  return n;
}

void Circuit::HA(Sig a, Sig b, Sig* s, Sig* c) {
  bool ca = sig_node(a) == 0, cb = sig_node(b) == 0;
  if (ca && cb) {
    bool va = sig_neg(a), vb = sig_neg(b);
    *s = (va != vb) ? SIG_ONE : SIG_ZERO;
    *c = (va && vb) ? SIG_ONE : SIG_ZERO;
    return;
  }
  if (ca || cb) {  // XOR(x,0)=x, XOR(x,1)=NOT x, AND(x,0)=0, AND(x,1)=x
    Sig x = ca ? b : a;
    bool k = sig_neg(ca ? a : b);
    *s = k ? NOT(x) : x;
    *c = k ? x : SIG_ZERO;
    return;
  }
  if (nand) {  // the sequence is explicit: argument evaluation order is unspecified
    const Sig t = NAND(a, b);
    const Sig u = NAND(a, t);
    const Sig v = NAND(b, t);
    *s = NAND(u, v);
    *c = NAND(t, t);
    n_xor++;
    n_and++;
    return;
  }
  uint32_t d = 1 + std::max(dep(a), dep(b));
  Product p;
  if (dep(b) > dep(a)) {
    p.a = b;
    p.b = a;
  } else {
    p.a = a;
    p.b = b;
  }
  p.is_or = false;
  p.is_add = false;
  p.is_nand = false;
  const uint64_t key = ((uint64_t)p.a << 32) | p.b;
  auto hit = memo_ha.find(key);
  if (hit != memo_ha.end()) {
    *s = products[hit->second].out_xor;
    *c = products[hit->second].out_and;
    return;
  }
  int32_t id = (int32_t)products.size();
  memo_ha[key] = id;
  products.push_back(p);
  uint32_t ns = new_node(d, id);
  uint32_t nc = new_node(d, id);
  products[id].out_xor = ns;
  products[id].out_and = nc;
  n_xor++;
  n_and++;
  *s = ns;
  *c = nc;
}

Sig Circuit::OR(Sig a, Sig b) {
  if (a == SIG_ONE || b == SIG_ONE) return SIG_ONE;
  if (a == SIG_ZERO) return b;
  if (b == SIG_ZERO) return a;
  if (nand) {
    n_or++;
    const Sig na = NOT(a);
    const Sig nb = NOT(b);
    return NAND(na, nb);
  }
  uint32_t d = 1 + std::max(dep(a), dep(b));
  Product p;
  if (dep(b) > dep(a)) {
    p.a = b;
    p.b = a;
  } else {
    p.a = a;
    p.b = b;
  }
  p.is_or = true;
  p.is_add = false;
  p.is_nand = false;
  p.out_and = 0;
  const uint64_t key = ((uint64_t)p.a << 32) | p.b;
  auto hit = memo_or.find(key);
  if (hit != memo_or.end()) return products[hit->second].out_xor;
  int32_t id = (int32_t)products.size();
  memo_or[key] = id;
  products.push_back(p);
  uint32_t n = new_node(d, id);
  products[id].out_xor = n;
  n_or++;
  return n;
}

Sig Circuit::XADD(Sig a, Sig b) {
  if (a == SIG_ONE || b == SIG_ONE) return SIG_ONE;
  if (a == SIG_ZERO) return b;
  if (b == SIG_ZERO) return a;
  uint32_t d = std::max(dep(a), dep(b));   // linear: no new multiplicative level
  Product p;
  if (dep(b) > dep(a)) {
    p.a = b;
    p.b = a;
  } else {
    p.a = a;
    p.b = b;
  }
  p.is_or = false;
  p.is_add = true;
  p.is_nand = false;
  p.out_and = 0;
  const uint64_t key = ((uint64_t)p.a << 32) | p.b;
  auto hit = memo_add.find(key);
  if (hit != memo_add.end()) return products[hit->second].out_xor;
  int32_t id = (int32_t)products.size();
  memo_add[key] = id;
  products.push_back(p);
  uint32_t n = new_node(d, id);
  products[id].out_xor = n;
  n_xadd++;
  return n;
}

void Circuit::FA(Sig a, Sig b, Sig c, Sig* s, Sig* co) {
  Sig s1, c1, c2;
  HA(a, b, &s1, &c1);
  HA(s1, c, s, &c2);
  *co = xcarry ? XADD(c1, c2) : OR(c1, c2);
}

std::vector<Sig> Circuit::ADD(const std::vector<Sig>& x, const std::vector<Sig>& y, Sig cin) {
  size_t F = x.size();
  std::vector<Sig> out(F);
  Sig carry;
  if (cin == SIG_ZERO)
    HA(x[0], y[0], &out[0], &carry);
  else
    FA(x[0], y[0], cin, &out[0], &carry);
  for (size_t i = 1; i < F; i++) FA(x[i], y[i], carry, &out[i], &carry);
  return out;  // carry out of the top bit is dropped (wrap mod 2^F)
}

std::vector<Sig> Circuit::SUB(const std::vector<Sig>& x, const std::vector<Sig>& y) {
  std::vector<Sig> ny(y.size());
  for (size_t i = 0; i < y.size(); i++) ny[i] = NOT(y[i]);
  return ADD(x, ny, SIG_ONE);
}

std::vector<Sig> Circuit::MUL(const std::vector<Sig>& x, int64_t w, uint32_t f) {
  const uint32_t F = (uint32_t)x.size();
  const uint32_t T = f + F;
  std::vector<Sig> xe(T);
  for (uint32_t j = 0; j < T; j++) xe[j] = x[std::min(j, F - 1)];
  const uint64_t wb = (uint64_t)w & (T >= 64 ? ~0ull : ((1ull << T) - 1));
  std::vector<std::vector<Sig>> col(T);
  for (uint32_t i = 0; i < T; i++)
    if ((wb >> i) & 1)
      for (uint32_t c = i; c < T; c++) col[c].push_back(xe[c - i]);
  std::vector<Sig> prod = wallace(std::move(col));
  return std::vector<Sig>(prod.begin() + f, prod.begin() + f + F);
}

std::vector<Sig> Circuit::MULE(const std::vector<Sig>& x, const std::vector<Sig>& y, uint32_t f) {
  const uint32_t F = (uint32_t)x.size();
  const uint32_t T = f + F;
  std::vector<Sig> xe(T), ye(T);
  for (uint32_t j = 0; j < T; j++) {
    xe[j] = x[std::min(j, F - 1)];
    ye[j] = y[std::min(j, F - 1)];
  }
  std::vector<std::vector<Sig>> col(T);
  for (uint32_t i = 0; i < T; i++)
    for (uint32_t c = i; c < T; c++) col[c].push_back(AND(xe[c - i], ye[i]));
  std::vector<Sig> prod = wallace(std::move(col));
  return std::vector<Sig>(prod.begin() + f, prod.begin() + f + F);
}

std::vector<Sig> Circuit::wallace(std::vector<std::vector<Sig>> col) {
  const uint32_t T = (uint32_t)col.size();
  auto tallest = [&]() {
    size_t h = 0;
    for (auto& v : col) h = std::max(h, v.size());
    return h;
  };
  while (tallest() > 2) {
    std::vector<std::vector<Sig>> sums(T), carries(T + 1);
    std::vector<Sig> pass(T, 0);
    std::vector<bool> has_pass(T, false);
    for (uint32_t c = 0; c < T; c++) {
      const auto& L = col[c];
      size_t g = 0;
      while (L.size() - g >= 3) {
        Sig s, cy;
        FA(L[g], L[g + 1], L[g + 2], &s, &cy);
        sums[c].push_back(s);
        carries[c + 1].push_back(cy);
        g += 3;
      }
      if (L.size() - g == 2) {
        Sig s, cy;
        HA(L[g], L[g + 1], &s, &cy);
        sums[c].push_back(s);
        carries[c + 1].push_back(cy);
      } else if (L.size() - g == 1) {
        pass[c] = L[g];
        has_pass[c] = true;
      }
    }
    for (uint32_t c = 0; c < T; c++) {
      std::vector<Sig> nc = sums[c];
      if (has_pass[c]) nc.push_back(pass[c]);
      nc.insert(nc.end(), carries[c].begin(), carries[c].end());
      col[c] = nc;
    }
  }
  std::vector<Sig> r0(T), r1(T);
  for (uint32_t c = 0; c < T; c++) {
    r0[c] = col[c].size() >= 1 ? col[c][0] : SIG_ZERO;
    r1[c] = col[c].size() >= 2 ? col[c][1] : SIG_ZERO;
  }
  return ADD(r0, r1, SIG_ZERO);
}

void twiddles(uint32_t N, uint32_t f, std::vector<int64_t>* wr, std::vector<int64_t>* wi) {
  wr->clear();
  wi->clear();
  const double pi = 3.14159265358979323846;
  for (uint32_t k = 0; k < N / 2; k++) {
    double ang = 2.0 * pi * (double)k / (double)N;
    wr->push_back((int64_t)std::floor(std::cos(ang) * (double)(1ull << f)));
    wi->push_back((int64_t)std::floor(-std::sin(ang) * (double)(1ull << f)));
  }
}

namespace {

using Word = std::vector<Sig>;
using Cplx = std::pair<Word, Word>;

uint32_t bitrev(uint32_t i, uint32_t bits) {
  uint32_t r = 0;
  for (uint32_t b = 0; b < bits; b++) {
    r = (r << 1) | (i & 1);
    i >>= 1;
  }
  return r;
}

// Twiddle of a butterfly: a plaintext pair (MUL) or an encrypted pair (MULE).
struct Twiddle {
  int64_t wr = 0, wi = 0;
  const Cplx* enc = nullptr;
};

Word mul_tw(Circuit* c, const Word& x, const Twiddle& w, bool real, uint32_t f) {
  if (w.enc) return c->MULE(x, real ? w.enc->first : w.enc->second, f);
  return c->MUL(x, real ? w.wr : w.wi, f);
}

void butterfly(Circuit* c, Cplx* u, Cplx* x, const Twiddle& w, uint32_t f) {
  // operands in the order t_r = xr Wr - xi Wi, t_i = xi Wr + xr Wi
  Word p0 = mul_tw(c, x->first, w, true, f);
  Word p1 = mul_tw(c, x->second, w, false, f);
  Word tr = c->SUB(p0, p1);
  Word p2 = mul_tw(c, x->second, w, true, f);
  Word p3 = mul_tw(c, x->first, w, false, f);
  Word ti = c->ADD(p2, p3, SIG_ZERO);
  Word top_r = c->ADD(u->first, tr, SIG_ZERO);
  Word top_i = c->ADD(u->second, ti, SIG_ZERO);
  Word bot_r = c->SUB(u->first, tr);
  Word bot_i = c->SUB(u->second, ti);
  *u = Cplx(top_r, top_i);
  *x = Cplx(bot_r, bot_i);
}

// table: encrypted twiddles W_M^k (k < M/2) or empty for plaintext constants
std::vector<Cplx> fft(Circuit* c, const std::vector<Cplx>& in, uint32_t f,
                      const std::vector<Cplx>& table) {
  const uint32_t N = (uint32_t)in.size();
  uint32_t logN = 0;
  while ((1u << logN) < N) logN++;
  std::vector<Twiddle> tw(N / 2);
  if (table.empty()) {
    std::vector<int64_t> wr, wi;
    twiddles(N, f, &wr, &wi);
    for (uint32_t t = 0; t < N / 2; t++) {
      tw[t].wr = wr[t];
      tw[t].wi = wi[t];
    }
  } else {
    const uint32_t M = 2 * (uint32_t)table.size();
    for (uint32_t t = 0; t < N / 2; t++) tw[t].enc = &table[t * (M / N)];
  }
  std::vector<Cplx> a(N);
  for (uint32_t i = 0; i < N; i++) a[i] = in[bitrev(i, logN)];
  for (uint32_t m = 2; m <= N; m *= 2) {
    uint32_t h = m / 2;
    for (uint32_t k = 0; k < N; k += m)
      for (uint32_t j = 0; j < h; j++) {
        butterfly(c, &a[k + j], &a[k + j + h], tw[j * (N / m)], f);
      }
  }
  return a;
}

bool pow2(uint32_t n) { return n >= 1 && (n & (n - 1)) == 0; }

}  // namespace

bool build_fft(Circuit* c, uint32_t N1, uint32_t N2, uint32_t F, uint32_t f) {
  if (!pow2(N1) || !pow2(N2) || F < 2 || F > 48 || f >= F) return false;
  if (c->enc_twiddle && f + 2 > F) return false;   // W^0 = 2^f must fit a signed word
  const uint32_t count = N1 * N2;
  auto input_word = [&]() {
    Word re(F), im(F);
    for (uint32_t b = 0; b < F; b++) re[b] = c->new_input();
    for (uint32_t b = 0; b < F; b++) im[b] = c->new_input();
    return Cplx(re, im);
  };
  std::vector<Cplx> s(count);
  for (uint32_t k = 0; k < count; k++) s[k] = input_word();
  std::vector<Cplx> table;
  if (c->enc_twiddle)
    for (uint32_t k = 0; k < std::max(N1, N2) / 2; k++) table.push_back(input_word());
  std::vector<Cplx> out;
  if (N2 == 1) {
    out = N1 > 1 ? fft(c, s, f, table) : s;
  } else {
    std::vector<Cplx> grid(count);
    for (uint32_t r = 0; r < N1; r++) {
      std::vector<Cplx> row(s.begin() + r * N2, s.begin() + (r + 1) * N2);
      std::vector<Cplx> res = N2 > 1 ? fft(c, row, f, table) : row;
      for (uint32_t j = 0; j < N2; j++) grid[r * N2 + j] = res[j];
    }
    out = grid;
    if (N1 > 1)
      for (uint32_t col = 0; col < N2; col++) {
        std::vector<Cplx> v(N1);
        for (uint32_t r = 0; r < N1; r++) v[r] = grid[r * N2 + col];
        std::vector<Cplx> res = fft(c, v, f, table);
        for (uint32_t r = 0; r < N1; r++) out[r * N2 + col] = res[r];
      }
  }
  for (auto& z : out) {
    c->outputs.insert(c->outputs.end(), z.first.begin(), z.first.end());
    c->outputs.insert(c->outputs.end(), z.second.begin(), z.second.end());
  }
  return true;
}

bool build_words(Circuit* c, uint32_t op, uint64_t count, uint32_t F, uint32_t f) {
  // a word's circuit has O((f + F)^2) nodes: keep the whole circuit (host
  // memory, 31-bit node ids) within 2^28 nodes of that order
  if (count == 0 || F < 2 || F > 48 || f >= F) return false;
  if (count * (uint64_t)(f + F) * (f + F) > (1ull << 28)) return false;
  if (op != SFFT_WORD_ADD && op != SFFT_WORD_SUB && op != SFFT_WORD_MUL) return false;
  for (uint64_t k = 0; k < count; k++) {
    Word x(F), y(F);
    for (uint32_t b = 0; b < F; b++) x[b] = c->new_input();
    for (uint32_t b = 0; b < F; b++) y[b] = c->new_input();
    Word r = op == SFFT_WORD_ADD ? c->ADD(x, y, SIG_ZERO)
           : op == SFFT_WORD_SUB ? c->SUB(x, y)
                                 : c->MULE(x, y, f);
    c->outputs.insert(c->outputs.end(), r.begin(), r.end());
  }
  return true;
}

bool build_refresh(Circuit* c, uint32_t n, uint32_t ell, uint64_t count) {
  const uint64_t rows = (uint64_t)n * ell + 1;
  uint32_t pb = 0;
  while ((1ull << pb) < rows) pb++;
  pb += 3;
  // one refresh has ~7 (n ell + 1) p nodes: keep the circuit within 2^28
  if (n == 0 || count == 0 || pb > ell || count * rows * pb * 7 > (1ull << 28)) return false;
  const uint32_t tau = ell - pb;
  std::vector<uint32_t> bk(rows);
  for (uint64_t r = 0; r < rows; r++) bk[r] = c->new_input();
  for (uint64_t i = 0; i < count; i++) {
    std::vector<std::vector<Sig>> col(pb);
    for (uint32_t k = 0; k < pb; k++) {
      col[k].push_back(c->SEL(0, (uint32_t)i, tau + k));
      for (uint32_t j = 1; j <= n; j++)
        for (uint32_t b = 0; b <= tau + k && b < ell; b++)
          col[k].push_back(c->SEL(1 + (j - 1) * ell + b, (uint32_t)i, j * ell + tau + k - b));
    }
    std::vector<Sig> S = c->wallace(std::move(col));
    Sig s, cy;
    c->HA(S[pb - 1], S[pb - 2], &s, &cy);
    c->outputs.push_back(s);
  }
  return true;
}

int build_circuit(Circuit* c, const CircuitSpec& spec, uint32_t flags) {
  if (!c->set_variant(flags))
    return fail(SFFT_EINVAL, "SFFT_PLAN_XCARRY and SFFT_PLAN_NAND are exclusive");
  if (spec.op == kOpRefresh) {
    if (!build_refresh(c, spec.n, spec.ell, spec.count))
      return fail(SFFT_EINVAL, "refresh needs n >= 1, count >= 1 with count (n ell + 1) "
                               "(log2(n ell + 1) + 3) <= 2^28 / 7, and ell >= "
                               "ceil(log2(n ell + 1)) + 3");
    return SFFT_OK;
  }
  if (spec.op == 0) {
    if (!build_fft(c, spec.N1, spec.N2, spec.F, spec.f))
      return fail(SFFT_EINVAL,
                  "N1, N2 must be powers of two, 2 <= F <= 48, f < F (f <= F - 2 with "
                  "encrypted twiddles)");
    return SFFT_OK;
  }
  if (!build_words(c, spec.op, spec.count, spec.F, spec.f))
    return fail(SFFT_EINVAL, "word op must be SFFT_WORD_ADD/SUB/MUL, count >= 1 with "
                             "count (f + F)^2 <= 2^28, "
                             "2 <= F <= 48, f < F");
  return SFFT_OK;
}

// ------------------------------------------------------------ noise bound

namespace {

// Minimal non-negative big integer: little-endian base 2^32.
struct Big {
  std::vector<uint32_t> d;
  static Big of(uint64_t v) {
    Big b;
    while (v) {
      b.d.push_back((uint32_t)v);
      v >>= 32;
    }
    return b;
  }
  // a ka + b kb in one pass (ka, kb < 2^32)
  static Big lin(const Big& a, uint64_t ka, const Big& b, uint64_t kb) {
    Big r;
    const size_t n = std::max(a.d.size(), b.d.size());
    r.d.reserve(n + 2);
    unsigned __int128 carry = 0;
    for (size_t i = 0; i < n; i++) {
      carry += (unsigned __int128)(i < a.d.size() ? a.d[i] : 0u) * ka;
      carry += (unsigned __int128)(i < b.d.size() ? b.d[i] : 0u) * kb;
      r.d.push_back((uint32_t)carry);
      carry >>= 32;
    }
    while (carry) {
      r.d.push_back((uint32_t)carry);
      carry >>= 32;
    }
    r.trim();
    return r;
  }
  void trim() {
    while (!d.empty() && d.back() == 0) d.pop_back();
  }
  uint32_t bits() const {
    if (d.empty()) return 0;
    uint32_t top = d.back(), b = 0;
    while (top) {
      b++;
      top >>= 1;
    }
    return (uint32_t)(d.size() - 1) * 32 + b;
  }
};

struct Code {
  int c0, c1, c2, c3;
};
constexpr Code kXor = {0, 1, 1, -2};
constexpr Code kAnd = {0, 0, 0, 1};
constexpr Code kOr = {0, 1, 1, -1};
constexpr Code kAdd = {0, 1, 1, 0};
constexpr Code kNand = {1, 0, 0, -1};

// Liveness: which products and nodes reach an output.
void liveness(const Circuit& c, std::vector<char>* live_node, std::vector<char>* live_prod) {
  live_node->assign(c.depth.size(), 0);
  live_prod->assign(c.products.size(), 0);
  for (Sig s : c.outputs) (*live_node)[sig_node(s)] = 1;
  for (int64_t p = (int64_t)c.products.size() - 1; p >= 0; p--) {
    const Product& g = c.products[p];
    bool l = (g.out_xor && (*live_node)[g.out_xor]) || (g.out_and && (*live_node)[g.out_and]);
    if (!l) continue;
    (*live_prod)[p] = 1;
    (*live_node)[sig_node(g.a)] = 1;
    (*live_node)[sig_node(g.b)] = 1;
  }
  (*live_node)[0] = 0;
}

}  // namespace

uint32_t noise_bits(const Circuit& c, const Shape& s) {
  std::vector<char> ln, lp;
  liveness(c, &ln, &lp);
  std::vector<Big> E(c.depth.size());
  Big fresh = Big::of((uint64_t)s.m * s.chi);
  for (uint32_t n : c.inputs) E[n] = fresh;
  for (const auto& kv : c.vin_of) E[kv.first] = fresh;   // worst case: selected
  uint32_t best = fresh.bits();
  for (size_t p = 0; p < c.products.size(); p++) {
    if (!lp[p]) continue;
    const Product& g = c.products[p];
    const Big& EA = E[sig_node(g.a)];
    const Big& EB = E[sig_node(g.b)];
    auto apply = [&](uint32_t node, Code k) {
      if (!node || !ln[node]) return;
      Big e = Big::lin(EA, (uint64_t)(std::abs(k.c1) + std::abs(k.c3)), EB,
                       (uint64_t)std::abs(k.c2) + (uint64_t)std::abs(k.c3) * s.Ng);
      best = std::max(best, e.bits());
      E[node] = e;
    };
    if (g.is_add) {
      apply(g.out_xor, kAdd);
    } else if (g.is_nand) {
      apply(g.out_xor, kNand);
    } else if (g.is_or) {
      apply(g.out_xor, kOr);
    } else {
      apply(g.out_xor, kXor);
      apply(g.out_and, kAnd);
    }
  }
  return best;
}

// -------------------------------------------------------------- compile

namespace {

// Coefficients on stored operands: a complemented B is absorbed first
// (c2 B~ = c2 P - c2 B; c3 BitDecomp(A~)(P - B) = c3 A~ - c3 BitDecomp(A~) B),
// then a complemented A in the linear term (c1 A~ = c1 P - c1 A); the kernel
// itself complements A before BitDecomp.
uint16_t adjusted(Code k, bool negA, bool negB) {
  if (negB) {
    k.c0 += k.c2;
    k.c2 = -k.c2;
    k.c1 += k.c3;
    k.c3 = -k.c3;
  }
  if (negA) {
    k.c0 += k.c1;
    k.c1 = -k.c1;
  }
  return pack_code(k.c0, k.c1, k.c2, k.c3);
}

}  // namespace

uint64_t level_cap(const CircuitSpec& spec) { return spec.op == kOpRefresh ? kRefreshLevelCap : 0; }

void compile(const Circuit& c, const Shape& s, Program* prog, uint64_t width_cap, uint32_t reuse_gap) {
  if (reuse_gap < 1) reuse_gap = 1;
  std::vector<char> ln, lp;
  liveness(c, &ln, &lp);
  const size_t nn = c.depth.size();
  std::vector<uint32_t> home(nn, REF_NONE);
  std::vector<uint32_t> last(nn, 0);
  // Schedule level of every node: a product runs in level 1 + max of its
  // inputs' levels; a linear gate runs after the products of the level of its
  // inputs (one level later for an input that is itself a linear output of
  // that level), and never before level 1.
  std::vector<uint32_t> sl(nn, 0);
  std::vector<uint32_t> plev(c.products.size(), 0);
  std::vector<char> lin_node(nn, 0);
  std::vector<uint64_t> width(2, 0);   // products per level so far
  uint32_t maxlev = 0;
  for (size_t p = 0; p < c.products.size(); p++) {
    if (!lp[p]) continue;
    const Product& g = c.products[p];
    const uint32_t na = sig_node(g.a), nb = sig_node(g.b);
    uint32_t lev;
    if (g.is_add)
      lev = std::max(1u, std::max(sl[na] + lin_node[na], sl[nb] + lin_node[nb]));
    else
      lev = 1 + std::max(sl[na], sl[nb]);
    if (!g.is_add) {
      if (width_cap)
        while (lev < width.size() && width[lev] >= width_cap) lev++;
      if (lev >= width.size()) width.resize(lev + 1, 0);
      width[lev]++;
    }
    plev[p] = lev;
    for (uint32_t node : {g.out_xor, g.out_and})
      if (node) {
        sl[node] = lev;
        lin_node[node] = g.is_add;
      }
    maxlev = std::max(maxlev, lev);
    last[na] = std::max(last[na], lev);
    last[nb] = std::max(last[nb], lev);
  }
  for (size_t i = 0; i < c.inputs.size(); i++) home[c.inputs[i]] = make_ref(REG_IN, (uint32_t)i);
  for (const auto& kv : c.vin_of) home[kv.first] = make_ref(REG_IN, c.vin[kv.second].input);

  // Outputs: a gate-produced, uncomplemented node lives directly in its first
  // output slot; everything else is materialised by a fix-up after the last
  // level (reads of fix-up sources count as uses at level maxlev + 1).
  prog->fix.clear();
  for (size_t o = 0; o < c.outputs.size(); o++) {
    Sig sg = c.outputs[o];
    uint32_t node = sig_node(sg);
    if (node != 0 && !sig_neg(sg) && c.producer[node] >= 0 && home[node] == REF_NONE) {
      home[node] = make_ref(REG_OUT, (uint32_t)o);
      continue;
    }
    FixDesc f{};
    f.dst = (uint32_t)o;
    f.src = node;  // node id for now, resolved below
    f.kind = node == 0 ? (sig_neg(sg) ? 3u : 2u) : (sig_neg(sg) ? 1u : 0u);
    prog->fix.push_back(f);
    if (node) last[node] = std::max(last[node], maxlev + 1);
  }

  // Group live gates by level: products first, then linear gates (each in
  // creation order, which is topological).
  std::vector<std::vector<uint32_t>> by_level(maxlev + 1), lin_level(maxlev + 1);
  for (size_t p = 0; p < c.products.size(); p++) {
    if (!lp[p]) continue;
    (c.products[p].is_add ? lin_level : by_level)[plev[p]].push_back((uint32_t)p);
  }
  std::vector<std::vector<uint32_t>> release(maxlev + reuse_gap + 1);
  std::vector<uint32_t> free_slots;
  uint32_t next_slot = 0;
  prog->desc.clear();
  prog->aux.clear();
  prog->patch.clear();
  prog->level_off.assign(1, 0);
  prog->lin_start.clear();
  prog->max_width = 0;
  uint64_t n_products = 0;
  for (uint32_t lev = 1; lev <= maxlev; lev++) {
    for (int phase = 0; phase < 2; phase++) {
      if (phase == 1) prog->lin_start.push_back(prog->desc.size());
      for (uint32_t p : phase ? lin_level[lev] : by_level[lev]) {
        const Product& g = c.products[p];
        for (uint32_t node : {g.out_xor, g.out_and}) {
          if (!node || !ln[node] || home[node] != REF_NONE) continue;
          uint32_t slot;
          if (!free_slots.empty()) {
            slot = free_slots.back();
            free_slots.pop_back();
          } else {
            slot = next_slot++;
          }
          home[node] = make_ref(REG_SCRATCH, slot);
          release[last[node] + reuse_gap - 1].push_back(node);   // free from level last + gap
        }
        GateDesc d;
        GateAux x;
        bool negA = sig_neg(g.a), negB = sig_neg(g.b);
        d.a = home[sig_node(g.a)];
        d.b = home[sig_node(g.b)];
        uint16_t k0, k1 = 0;
        if (g.is_add || g.is_nand) {
          d.o0 = ln[g.out_xor] ? home[g.out_xor] : REF_NONE;
          d.o1 = REF_NONE;
          k0 = adjusted(g.is_add ? kAdd : kNand, negA, negB);
        } else if (g.is_or) {
          d.o0 = ln[g.out_xor] ? home[g.out_xor] : REF_NONE;
          d.o1 = REF_NONE;
          k0 = adjusted(kOr, negA, negB);
        } else {
          d.o0 = (g.out_xor && ln[g.out_xor]) ? home[g.out_xor] : REF_NONE;
          d.o1 = (g.out_and && ln[g.out_and]) ? home[g.out_and] : REF_NONE;
          k0 = adjusted(kXor, negA, negB);
          k1 = adjusted(kAnd, negA, negB);
        }
        x.code = (uint32_t)k0 | ((uint32_t)k1 << 16);
        x.flags = (negA && !g.is_add) ? 1u : 0u;   // complement A before BitDecomp (products only)
        auto va = c.vin_of.find(sig_node(g.a)), vb = c.vin_of.find(sig_node(g.b));
        if (va != c.vin_of.end() || vb != c.vin_of.end()) {
          PatchDesc pd{};
          pd.gate = (uint32_t)prog->desc.size();
          pd.code = x.code;
          pd.a_ct = pd.b_ct = REF_NONE;
          if (va != c.vin_of.end()) {
            pd.a_ct = c.vin[va->second].src_ct;
            pd.a_pos = c.vin[va->second].src_pos;
          }
          if (vb != c.vin_of.end()) {
            pd.b_ct = c.vin[vb->second].src_ct;
            pd.b_pos = c.vin[vb->second].src_pos;
          }
          prog->patch.push_back(pd);
        }
        prog->desc.push_back(d);
        prog->aux.push_back(x);
      }
    }
    n_products += by_level[lev].size();
    prog->level_off.push_back(prog->desc.size());
    prog->max_width = std::max<uint64_t>(prog->max_width, by_level[lev].size());
    for (uint32_t node : release[lev]) {
      uint32_t r = home[node];
      if ((r >> 30) == REG_SCRATCH) free_slots.push_back(r & SLOT_MASK);
    }
  }
  for (auto& f : prog->fix) f.src = f.src ? home[f.src] : 0;
  prog->n_inputs = c.inputs.size();
  prog->n_outputs = c.outputs.size();
  prog->scratch_slots = next_slot;
  prog->products = n_products;
  prog->noise_bits = noise_bits(c, s);
  prog->noise_ok = prog->noise_bits <= s.ell - 2;
}

bool persistent_schedule(const Program& m, std::vector<uint32_t>* glev, std::vector<uint32_t>* dep_a,
                         std::vector<uint32_t>* dep_b, std::vector<uint32_t>* lwidth) {
  const uint32_t levels = (uint32_t)(m.level_off.size() - 1);
  for (uint32_t l = 0; l < levels; l++)
    if (m.lin_start[l] != m.level_off[l + 1]) return false;
  const uint64_t n = m.desc.size();
  glev->assign(n, 0);
  dep_a->assign(n, 0xFFFFFFFFu);
  dep_b->assign(n, 0xFFFFFFFFu);
  lwidth->assign(levels, 0);
  std::unordered_map<uint32_t, uint32_t> writer;   // slot reference -> last gate that wrote it
  writer.reserve(2 * n);
  auto dep_of = [&](uint32_t ref) -> uint32_t {
    if ((ref >> 30) == REG_IN) return 0xFFFFFFFFu;   // a program input
    auto it = writer.find(ref);
    return it == writer.end() ? 0xFFFFFFFFu : it->second;
  };
  for (uint32_t l = 0; l < levels; l++) {
    (*lwidth)[l] = (uint32_t)(m.level_off[l + 1] - m.level_off[l]);
    for (uint64_t g = m.level_off[l]; g < m.level_off[l + 1]; g++) {
      (*glev)[g] = l;
      (*dep_a)[g] = dep_of(m.desc[g].a);
      (*dep_b)[g] = dep_of(m.desc[g].b);
    }
    // writes after every read of the level (a level never writes what it reads)
    for (uint64_t g = m.level_off[l]; g < m.level_off[l + 1]; g++) {
      if (m.desc[g].o0 != REF_NONE) writer[m.desc[g].o0] = (uint32_t)g;
      if (m.desc[g].o1 != REF_NONE) writer[m.desc[g].o1] = (uint32_t)g;
    }
  }
  return true;
}

}  // namespace sfft
