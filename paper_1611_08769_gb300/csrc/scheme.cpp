// GSW'13 client side on the host: KeyGen, Enc (compressed), Dec, and the
// fixed-point encoding of signals.
//
// Compressed GSW (a ciphertext C is kept as C' = BitDecomp^-1(C), Ng rows of
// n+1 elements of Z_q):
//   KeyGen: t <- Z_q^n, s = (1, -t), B <- Z_q^{m x n}, e <- [-chi, chi]^m,
//           A = [B t + e | B]
//   Enc:    C' = R A + mu P (mod q), R in {0,1}^{Ng x m}, P[j ell + b][j] = 2^b
//   Dec:    x = <C'_{ell-1}, s> (mod q); mu = 1 iff q/4 <= x < 3q/4
// The paper cites the scheme for these steps (Sec. 3; Lemmas 1-2).
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "common.h"
#include "rng.h"
#include "scheme.h"

namespace sfft {

namespace {
thread_local std::string g_err;
}

void set_error(const std::string& msg) { g_err = msg; }
int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int make_shape(const sfft_params* p, Shape* s, bool need_square_key) {
  if (!p) return fail(SFFT_EINVAL, "params is NULL");
  if (p->ell == 0 || p->ell % 32 != 0 || p->ell > 8192)
    return fail(SFFT_EPARAM, "ell must be a multiple of 32 in [32, 8192]");
  if (p->n == 0 || p->n > 64) return fail(SFFT_EPARAM, "n must be in [1, 64]");
  if (p->m == 0) return fail(SFFT_EPARAM, "m must be positive");
  s->n = p->n;
  s->ell = p->ell;
  s->m = p->m;
  s->chi = p->chi;
  s->L = p->ell / 32;
  s->NP1 = p->n + 1;
  s->W = s->NP1 * s->L;
  s->Ng = s->NP1 * p->ell;
  s->ctw = (uint64_t)s->Ng * s->W;
  if (need_square_key && s->m != s->Ng)
    return fail(SFFT_EPARAM, "device encryption needs m == (n+1)*ell");
  return SFFT_OK;
}

// --------------------------------------------------- multi-limb mod 2^ell

namespace {

using Limbs = std::vector<uint32_t>;

Limbs zq_from_stream(uint64_t state, uint64_t index, uint32_t L) {
  const uint32_t W64 = (L + 1) / 2;
  Limbs v(L);
  for (uint32_t w = 0; w < W64; w++) {
    uint64_t x = stream_out(state, index * W64 + w);
    v[2 * w] = (uint32_t)x;
    if (2 * w + 1 < L) v[2 * w + 1] = (uint32_t)(x >> 32);
  }
  return v;
}

Limbs mulmod(const Limbs& a, const Limbs& b) {
  const size_t L = a.size();
  std::vector<uint64_t> acc(L + 1, 0);
  Limbs r(L, 0);
  for (size_t i = 0; i < L; i++) {
    uint64_t carry = 0;
    for (size_t j = 0; i + j < L; j++) {
      uint64_t t = (uint64_t)a[i] * b[j] + r[i + j] + carry;
      r[i + j] = (uint32_t)t;
      carry = t >> 32;
    }
  }
  return r;
}

void addmod(Limbs* a, const Limbs& b) {
  uint64_t carry = 0;
  for (size_t i = 0; i < a->size(); i++) {
    uint64_t t = (uint64_t)(*a)[i] + b[i] + carry;
    (*a)[i] = (uint32_t)t;
    carry = t >> 32;
  }
}

Limbs small_signed(int64_t v, uint32_t L) {  // v mod 2^ell
  Limbs r(L, v < 0 ? 0xFFFFFFFFu : 0u);
  r[0] = (uint32_t)(uint64_t)v;
  if (L > 1) r[1] = (uint32_t)((uint64_t)v >> 32);
  return r;
}

Limbs negmod(const Limbs& a) {
  Limbs r(a.size());
  uint64_t carry = 1;
  for (size_t i = 0; i < a.size(); i++) {
    uint64_t t = (uint64_t)(~a[i]) + carry;
    r[i] = (uint32_t)t;
    carry = t >> 32;
  }
  return r;
}

}  // namespace

// ------------------------------------------------------------------ keys

struct KeysImpl {
  Shape s;
  std::vector<Limbs> t, sk;   // secret t and s = (1, -t)
  std::vector<uint32_t> A;    // m x (n+1) x L
  std::vector<int64_t> e;
};

}  // namespace sfft

struct sfft_keys {
  sfft::KeysImpl k;
};

using namespace sfft;

extern "C" {

const char* sfft_last_error(void) { return g_err.c_str(); }

uint64_t sfft_ct_words(const sfft_params* p) {
  Shape s;
  if (make_shape(p, &s, false) != SFFT_OK) return 0;
  return s.ctw;
}

int sfft_keygen(const sfft_params* p, uint64_t seed, sfft_keys** out) {
  if (!out) return fail(SFFT_EINVAL, "out is NULL");
  Shape s;
  int rc = make_shape(p, &s, false);
  if (rc) return rc;
  sfft_keys* K = new (std::nothrow) sfft_keys;
  if (!K) return fail(SFFT_ENOMEM, "host allocation failed");
  KeysImpl& k = K->k;
  k.s = s;
  const uint64_t kt = domain_key(seed, kDomT), kb = domain_key(seed, kDomB),
                 ke = domain_key(seed, kDomE);
  for (uint32_t j = 0; j < s.n; j++) k.t.push_back(zq_from_stream(kt, j, s.L));
  k.sk.push_back(small_signed(1, s.L));
  for (uint32_t j = 0; j < s.n; j++) k.sk.push_back(negmod(k.t[j]));
  k.A.assign((uint64_t)s.m * s.NP1 * s.L, 0);
  const uint64_t width = 2ull * s.chi + 1;
  for (uint32_t r = 0; r < s.m; r++) {
    int64_t er = (int64_t)(stream_out(ke, r) % width) - (int64_t)s.chi;
    k.e.push_back(er);
    Limbs b0 = small_signed(er, s.L);
    for (uint32_t j = 0; j < s.n; j++) {
      Limbs bj = zq_from_stream(kb, (uint64_t)r * s.n + j, s.L);
      addmod(&b0, mulmod(bj, k.t[j]));
      std::memcpy(&k.A[((uint64_t)r * s.NP1 + 1 + j) * s.L], bj.data(), 4 * s.L);
    }
    std::memcpy(&k.A[(uint64_t)r * s.NP1 * s.L], b0.data(), 4 * s.L);
  }
  *out = K;
  return SFFT_OK;
}

void sfft_keys_free(sfft_keys* k) { delete k; }

int sfft_keys_public(const sfft_keys* k, uint32_t* h_out, uint64_t cap_words) {
  if (!k || !h_out) return fail(SFFT_EINVAL, "null argument");
  if (cap_words < k->k.A.size()) return fail(SFFT_EINVAL, "output too small");
  std::memcpy(h_out, k->k.A.data(), 4 * k->k.A.size());
  return SFFT_OK;
}

int sfft_key_bits(const sfft_keys* K, uint8_t* h_bits, uint64_t cap) {
  if (!K || !h_bits) return fail(SFFT_EINVAL, "null argument");
  const Shape& s = K->k.s;
  const uint64_t rows = (uint64_t)s.n * s.ell + 1;
  if (cap < rows) return fail(SFFT_EINVAL, "output too small: n ell + 1 bytes needed");
  h_bits[0] = 1;
  for (uint32_t j = 1; j <= s.n; j++)
    for (uint32_t b = 0; b < s.ell; b++)
      h_bits[1 + (uint64_t)(j - 1) * s.ell + b] = (K->k.sk[j][b / 32] >> (b % 32)) & 1;
  return SFFT_OK;
}

int sfft_encrypt_bits(const sfft_keys* K, const double* h_re, const double* h_im, uint64_t count,
                      uint32_t F, uint32_t f, uint64_t enc_seed, uint32_t* h_ct_out) {
  if (!K || !h_re || !h_ct_out) return fail(SFFT_EINVAL, "null argument");
  if (F < 2 || F > 48 || f >= F) return fail(SFFT_EPARAM, "need 2 <= F <= 48 and f < F");
  const KeysImpl& k = K->k;
  const Shape& s = k.s;
  std::vector<uint8_t> bits;
  encode_signal(h_re, h_im, count, F, f, &bits);
  const uint64_t rbits = (uint64_t)s.Ng * s.m;
  std::vector<uint64_t> acc(s.W);
  for (uint64_t c = 0; c < bits.size(); c++) {
    const uint64_t st = ct_stream(enc_seed, c);
    uint32_t* ct = h_ct_out + c * s.ctw;
    for (uint32_t i = 0; i < s.Ng; i++) {
      std::fill(acc.begin(), acc.end(), 0);
      for (uint32_t kk = 0; kk < s.m; kk++) {
        uint64_t bi = (uint64_t)i * s.m + kk;
        if (!((stream_out(st, bi >> 6) >> (bi & 63)) & 1)) continue;
        const uint32_t* arow = &k.A[(uint64_t)kk * s.W];
        for (uint32_t w = 0; w < s.W; w++) acc[w] += arow[w];
      }
      if (bits[c]) acc[(i / s.ell) * s.L + (i % s.ell) / 32] += 1ull << (i % 32);
      for (uint32_t j = 0; j < s.NP1; j++) {  // carry within each element, drop the top
        uint64_t carry = 0;
        for (uint32_t l = 0; l < s.L; l++) {
          uint64_t v = acc[j * s.L + l] + carry;
          ct[(uint64_t)i * s.W + j * s.L + l] = (uint32_t)v;
          carry = v >> 32;
        }
      }
    }
    (void)rbits;
  }
  return SFFT_OK;
}

int sfft_decrypt(const sfft_keys* K, const uint32_t* h_rows, uint64_t row_stride_words,
                 uint64_t count, uint32_t F, uint32_t f, double* h_re, double* h_im,
                 int64_t* h_raw) {
  if (!K || !h_rows) return fail(SFFT_EINVAL, "null argument");
  if (F < 2 || F > 48 || f >= F) return fail(SFFT_EPARAM, "need 2 <= F <= 48 and f < F");
  const KeysImpl& k = K->k;
  const Shape& s = k.s;
  for (uint64_t smp = 0; smp < count; smp++) {
    for (uint32_t part = 0; part < 2; part++) {
      uint64_t word = 0;
      for (uint32_t b = 0; b < F; b++) {
        const uint32_t* row = h_rows + ((smp * 2 + part) * F + b) * row_stride_words;
        Limbs x(s.L, 0);
        for (uint32_t j = 0; j < s.NP1; j++) {
          Limbs cj(row + j * s.L, row + (j + 1) * s.L);
          addmod(&x, mulmod(cj, k.sk[j]));
        }
        uint32_t top2 = (x[s.L - 1] >> 30) & 3u;   // x in [q/4, 3q/4) <=> top bits 01 or 10
        if (top2 == 1u || top2 == 2u) word |= 1ull << b;
      }
      int64_t v = (int64_t)(word << (64 - F)) >> (64 - F);
      if (h_raw) h_raw[smp * 2 + part] = v;
      double val = std::ldexp((double)v, -(int)f);
      if (part == 0 && h_re) h_re[smp] = val;
      if (part == 1 && h_im) h_im[smp] = val;
    }
  }
  return SFFT_OK;
}

}  // extern "C"

namespace sfft {

void encode_signal(const double* re, const double* im, uint64_t count, uint32_t F, uint32_t f,
                   std::vector<uint8_t>* bits) {
  bits->assign(count * 2 * F, 0);
  const uint64_t mask = (F >= 64) ? ~0ull : ((1ull << F) - 1);
  for (uint64_t k = 0; k < count; k++)
    for (uint32_t part = 0; part < 2; part++) {
      double x = part == 0 ? re[k] : (im ? im[k] : 0.0);
      int64_t raw = (int64_t)std::floor(std::ldexp(x, (int)f));
      uint64_t u = (uint64_t)raw & mask;
      for (uint32_t b = 0; b < F; b++) (*bits)[(k * 2 + part) * F + b] = (u >> b) & 1;
    }
}

}  // namespace sfft
