// Canonical FFT gate circuit -> levelised device program.
//
// The circuit follows the paper's construction (Sec. 4, Lemmas 3-9): half
// adders (XOR + AND sharing one ciphertext product), full adders as two half
// adders and an OR (Lemma 6, Fig. 3), ripple-carry ADD and SUB = ADD(x, NOT y,
// carry 1), Wallace-tree constant multiplication with sign extension to
// T = f + F bits keeping bits [f, f+F) (Lemmas 8-9), radix-2 DIT butterflies
// on the bit-reversed signal, and row-then-column 2-D transforms.
//
// Canonical choices that fix every ciphertext bit (shared with any other
// implementation of the same circuit):
//  * the bit-decomposed operand A of a product is the input of strictly
//    greater multiplicative depth, ties keep the gate's first argument;
//  * gates with a trivial-constant input are folded (bit-exact in GSW);
//  * Wallace stages: per column FAs over consecutive triples, an HA over a
//    remaining pair, a lone wire passes; new column = sums, passed wire,
//    carries from below; repeat until every column has at most 2 wires.
//
// NOT gates never reach the device: a signal carries a complement bit, the
// kernel complements A before BitDecomp, and a complemented B is absorbed
// into the gate's coefficients (BitDecomp(A)(P - B) = A - BitDecomp(A) B).
//
// Variant (Circuit::xcarry): the full adder's two carries are never both 1
// (c1 = 1 forces s1 = 0, hence c2 = 0), so its carry is their sum, a linear
// gate XADD = (0, 1, 1, 0) with no ciphertext product whose noise adds
// instead of growing by Ng. XADD folds like OR (a constant 1 on one side
// forces the other carry to 0). For the operand rule it is linear (depth =
// max of its inputs); on the device it runs after the products of its
// schedule level.
//
// Encrypted-operand multiplier (MULE, a variant: the paper multiplies by
// plaintext constants, whose bits show through the Wallace tree, Sec. 4):
// both words sign-extended to T = f + F bits, every row i < T present, column
// c >= i receiving AND(x_ext[c-i], y_ext[i]); the same Wallace stages and
// final ADD_T as MUL; bits [f, f+F). With Circuit::enc_twiddle the FFT takes
// one table of encrypted twiddles W_M^k, k < M/2, M = max(N1, N2), as inputs
// after the signal; a length-n transform uses entry t M/n for W_n^t.
//
// NAND-only variant (Circuit::nand, the paper's literal construction, Lemma
// 4): constants fold first as above; every remaining gate is made of GSW NAND
// gates (1, 0, 0, -1), one product each: NOT a = NAND(a, a), AND = NOT(NAND),
// OR = NAND(NOT a, NOT b), and a half adder t = NAND(a, b), XOR =
// NAND(NAND(a, t), NAND(b, t)), AND = NAND(t, t). No complement bits.
#pragma once

#include <cstdint>
#include <unordered_map>
#include <vector>

#include "common.h"

namespace sfft {

// A signal: node id (0 = the constant zero) and a complement bit (bit 31).
using Sig = uint32_t;
constexpr Sig SIG_ZERO = 0u;
constexpr Sig SIG_ONE = 0x80000000u;
inline uint32_t sig_node(Sig s) { return s & 0x7FFFFFFFu; }
inline bool sig_neg(Sig s) { return (s >> 31) != 0; }

struct Product {
  Sig a, b;          // A (bit-decomposed) and B, already ordered by the depth rule
  uint32_t out_xor;  // node of the XOR output (HA), the OR or the XADD output; 0 = none
  uint32_t out_and;  // node of the AND output (HA only); 0 = none
  bool is_or;
  bool is_add;       // linear exclusive sum (XADD): no ciphertext product
  bool is_nand;      // GSW NAND gate (NAND-only variant)
};

// A selected bootstrapping-key wire of a refresh circuit: beta * input, with
// beta read at run time from a refreshed ciphertext (src_ct, bit src_pos of
// its row ell - 1, counted over the row's n + 1 elements of ell bits).
struct VInput {
  uint32_t input, src_ct, src_pos;
};

struct Circuit {
  std::vector<uint32_t> depth;     // per node; node 0 = constant zero
  std::vector<int32_t> producer;   // per node: product index or -1 (input/const)
  std::vector<Product> products;
  std::vector<uint32_t> inputs;    // input nodes in ciphertext order
  std::vector<Sig> outputs;        // output signals in ciphertext order
  uint64_t n_and = 0, n_xor = 0, n_or = 0, n_not = 0, n_xadd = 0;   // logical gates before pruning
  bool xcarry = false;             // full-adder carry as XADD instead of OR
  bool nand = false;               // every gate made of NAND gates
  bool enc_twiddle = false;        // FFT twiddles are encrypted inputs (MULE)
  // Common subexpressions: identical (kind, A, B) gates give identical
  // ciphertexts, so each is computed once (bit-exact).
  std::unordered_map<uint64_t, int32_t> memo_ha, memo_or, memo_add, memo_nand;
  std::vector<VInput> vin;                          // selected inputs (refresh)
  std::unordered_map<uint32_t, uint32_t> vin_of;    // node -> index into vin

  // Selects the variant from plan flags (SFFT_PLAN_XCARRY, SFFT_PLAN_NAND,
  // SFFT_PLAN_ENC_TWIDDLE); false if both gate variants are set.
  bool set_variant(uint32_t flags);

  uint32_t new_node(uint32_t d, int32_t prod);
  uint32_t new_input();
  uint32_t dep(Sig s) const { return depth[sig_node(s)]; }

  Sig NOT(Sig a);
  Sig AND(Sig a, Sig b);    // the AND output of a half adder (NAND-only: NOT(NAND))
  void HA(Sig a, Sig b, Sig* s, Sig* c);
  Sig OR(Sig a, Sig b);
  Sig XADD(Sig a, Sig b);
  Sig NAND(Sig a, Sig b);   // one GSW NAND gate on two non-constant signals
  // beta * inputs[input] with beta a run-time bit of a refreshed ciphertext:
  // a depth-0 leaf, never folded, never shared.
  Sig SEL(uint32_t input, uint32_t src_ct, uint32_t src_pos);
  void FA(Sig a, Sig b, Sig c, Sig* s, Sig* co);
  std::vector<Sig> ADD(const std::vector<Sig>& x, const std::vector<Sig>& y, Sig cin);
  std::vector<Sig> SUB(const std::vector<Sig>& x, const std::vector<Sig>& y);
  std::vector<Sig> MUL(const std::vector<Sig>& x, int64_t w, uint32_t f);
  std::vector<Sig> MULE(const std::vector<Sig>& x, const std::vector<Sig>& y, uint32_t f);
  // Wallace stages on column lists, then ADD_T of the two rows (T = columns).
  std::vector<Sig> wallace(std::vector<std::vector<Sig>> col);
};

// Builds the circuit of a 1-D (N2 == 1) or 2-D FFT. Throws nothing; returns
// false on invalid sizes (and f > F - 2 with encrypted twiddles).
bool build_fft(Circuit* c, uint32_t N1, uint32_t N2, uint32_t F, uint32_t f);

// count independent word operations (SFFT_WORD_ADD / SUB / MUL) on pairs of
// F-bit words: word k's x at inputs (2k) F + b, y at (2k + 1) F + b, result
// at outputs k F + b. false on invalid sizes.
bool build_words(Circuit* c, uint32_t op, uint64_t count, uint32_t F, uint32_t f);

// Refresh of count ciphertexts by homomorphic decryption of row ell - 1:
// inputs are the bootstrapping key (encryptions of sigma_0 = 1 and of bit b
// of s_j = -t_j mod q, j = 1..n, in that order); for each refreshed
// ciphertext i the p-bit sum S = sum_r K'_r sigma_r (mod 2^p), p =
// ceil(log2(n ell + 1)) + 3, K'_r = floor(K_r / 2^(ell - p)), K_0 = c_0,
// K_{j,b} = c_j 2^b mod q: column k gets SEL(sigma_r) selected by bit k of
// K'_r (bit ell - p + k - b of c_j, left out where that index is negative),
// Wallace stages and ADD_p; output i = XOR(S_{p-1}, S_{p-2}).
bool build_refresh(Circuit* c, uint32_t n, uint32_t ell, uint64_t count);
constexpr uint32_t kOpRefresh = 0x100;
constexpr uint64_t kRefreshLevelCap = 4096;   // products per level of a refresh program

// What a plan evaluates: an FFT (op 0), count word operations (SFFT_WORD_*)
// or count refreshes (kOpRefresh, at parameters n, ell).
struct CircuitSpec {
  uint32_t op = 0;
  uint32_t N1 = 1, N2 = 1;
  uint64_t count = 0;
  uint32_t F = 0, f = 0;
  uint32_t n = 0, ell = 0;
};

// Selects the variant from flags and builds the circuit; SFFT_OK or the
// error (recorded as the last error).
int build_circuit(Circuit* c, const CircuitSpec& spec, uint32_t flags);

// Quantised twiddles W_N^k = exp(-2 pi i k / N), k < N/2, floor to 2^-f.
void twiddles(uint32_t N, uint32_t f, std::vector<int64_t>* wr, std::vector<int64_t>* wi);

// Device program of a circuit for fixed scheme parameters.
struct Program {
  std::vector<GateDesc> desc;      // all gates, level by level
  std::vector<GateAux> aux;
  // level l = [level_off[l], level_off[l+1]): its products, then from
  // lin_start[l] on the linear gates (XADD) that run after them
  std::vector<uint64_t> level_off;
  std::vector<uint64_t> lin_start;
  std::vector<FixDesc> fix;        // output fix-ups
  std::vector<PatchDesc> patch;    // gates with selected operands (refresh)
  uint64_t n_inputs = 0, n_outputs = 0, scratch_slots = 0, products = 0;
  uint64_t max_width = 0;
  uint32_t noise_bits = 0;
  bool noise_ok = false;
};

// Prunes dead gates, levelises, allocates scratch slots with reuse after last
// use, and computes the static noise bound for the given parameters.
// width_cap > 0 bounds the products of a level: a product whose inputs are
// ready at level l runs at the first level >= l with room (creation order),
// which bounds the ciphertexts alive at once for circuits whose ready set is
// very wide (refresh). A scratch slot last read at level l is reused from
// level l + reuse_gap on (1: the next level; 2 for programs whose levels
// overlap by one on the device, the persistent batch).
void compile(const Circuit& c, const Shape& s, Program* prog, uint64_t width_cap = 0,
             uint32_t reuse_gap = 1);

// The persistent form's schedule of a compiled program (one launch across
// levels): each gate's level, the gates that last wrote its two operands
// before its level (0xFFFFFFFF: a program input), and each level's width. A
// gate may start once both producers are done and every gate two levels up
// is done; with reuse_gap 2 that window also orders every slot's reuse after
// its last read. False (nothing written) for programs with linear gates.
bool persistent_schedule(const Program& m, std::vector<uint32_t>* glev, std::vector<uint32_t>* dep_a,
                         std::vector<uint32_t>* dep_b, std::vector<uint32_t>* lwidth);

// The level width cap a plan of this kind compiles with (0: none).
uint64_t level_cap(const CircuitSpec& spec);

// Bit length of the largest static noise bound of the circuit's live wires
// (fresh ciphertext m * chi; gate (|c1|+|c3|) E_A + (|c2| + |c3| Ng) E_B).
uint32_t noise_bits(const Circuit& c, const Shape& s);

}  // namespace sfft
