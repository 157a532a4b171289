/*
 * sfft.h -- C ABI of the GB300 encrypted-FFT library.
 *
 * The library evaluates the paper's secure FFT: a radix-2 FFT over
 * bit-wise GSW-encrypted two's-complement fixed-point words, computed as a
 * circuit of homomorphic gates (Sec. 4) on one GPU. The calls follow the
 * paper's client/server workflow (Sec. 1, Fig. 1): key generation (step 1),
 * encryption of the signal bit by bit (step 2), evaluation of the FFT on the
 * server (step 4) and decryption (step 6).
 *
 * Conventions (every call):
 *  - Returns SFFT_OK (0) or a negative SFFT_E* code; sfft_last_error() gives
 *    a thread-local message for the last failure on the calling thread.
 *  - Pointers named h_* are host memory, d_* are device memory on the
 *    current CUDA device; neither is retained after the call returns.
 *  - Opaque handles (sfft_keys, sfft_plan, sfft_batch, sfft_server) are
 *    owned by the library and released with the matching *_free call. A plan
 *    or batch lives on the CUDA device current when it was created; evaluating
 *    it with another device current fails with EINVAL.
 *  - Scheme parameters: q = 2^ell with ell a multiple of 32; Ng = (n+1) ell.
 *    A ciphertext is stored compressed, C' = BitDecomp^-1(C): Ng rows of
 *    (n+1) elements of Z_q, each as L = ell/32 uint32 limbs, least
 *    significant limb first, row-major -- sfft_ct_words() words in all.
 *    Read as a little-endian bit string, row i is row i of the N x N binary
 *    GSW matrix (Sec. 3; Sec. 7 gives the N^2 ciphertext size).
 *  - Signals: sample k of a signal occupies ciphertexts (2k + part) * F + b
 *    for part 0 (real) / 1 (imaginary) and bit b = 0 .. F-1 (LSB first).
 *    2-D signals are N1 x N2 images, sample k = r * N2 + c.
 *  - Arithmetic wraps mod 2^F (two's complement); overflow is not an error.
 *  - Device calls are asynchronous on the given CUDA stream (NULL = legacy
 *    default stream) unless stated otherwise.
 */
#ifndef SFFT_H
#define SFFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  SFFT_OK = 0,
  SFFT_EINVAL = -1,   /* bad argument (null pointer, size, non power of two) */
  SFFT_ENOMEM = -2,   /* host or device allocation failed / budget exceeded */
  SFFT_ECUDA = -3,    /* a CUDA call failed */
  SFFT_ETIMEOUT = -4, /* a bounded wait ran out */
  SFFT_EPARAM = -5,   /* parameters unsupported or inconsistent (n, ell, F, f) */
  SFFT_EBUSY = -6,    /* resource in use */
  SFFT_ENOTFOUND = -7 /* unknown ticket */
};

/* GSW'13 parameters (Sec. 3 names the scheme but not its parameters).
 * n: LWE dimension; ell: log2 q (multiple of 32); m: rows of the public key
 * (the device paths need m == Ng); chi: error bound, e uniform in [-chi, chi]
 * (0 = noise-free toy parameters). */
typedef struct sfft_params {
  uint32_t n, ell, m, chi;
} sfft_params;

typedef struct sfft_keys sfft_keys;
typedef struct sfft_plan sfft_plan;
typedef struct sfft_batch sfft_batch;
typedef struct sfft_server sfft_server;

const char* sfft_last_error(void);
const char* sfft_version(void);
/* Running count of kernel launches this library has issued in the process
 * (graph replays excluded: they re-run launches counted at capture). */
uint64_t sfft_launch_count(void);

/* Words (uint32) of one compressed ciphertext: Ng * (n+1) * ell/32. */
uint64_t sfft_ct_words(const sfft_params* p);

/* ---------------------------------------------------------------- client */

/* Step 1, KeyGen (GSW'13 Sec. 3): t <- Z_q^n, s = (1, -t), B <- Z_q^{m x n},
 * e <- [-chi, chi]^m, A = [B t + e | B]. All randomness is the counter-based
 * SplitMix64 stream of ``seed`` (domains t = 1, B = 2, e = 3). Host only. */
int sfft_keygen(const sfft_params* p, uint64_t seed, sfft_keys** out);
void sfft_keys_free(sfft_keys* k);

/* Copies the public matrix A (m x (n+1) elements, limb layout as a
 * ciphertext) to h_out (cap_words >= m*(n+1)*ell/32). */
int sfft_keys_public(const sfft_keys* k, uint32_t* h_out, uint64_t cap_words);

/* Step 2, Enc of a fixed-point signal (Sec. 4 fixed point; Sec. 5
 * truncation): raw = floor(x * 2^f) mod 2^F for every sample, then every
 * bit mu is encrypted as C' = R A + mu P (mod q), R the Ng x m binary matrix
 * drawn from stream domain 4 for ciphertext index (2k + part) * F + b.
 * h_im may be NULL (imaginary part 0). Writes count*2*F ciphertexts to
 * h_ct_out (host). CPU implementation, for small parameters. */
int sfft_encrypt_bits(const sfft_keys* k, const double* h_re, const double* h_im,
                      uint64_t count, uint32_t F, uint32_t f, uint64_t enc_seed,
                      uint32_t* h_ct_out);

/* Same ciphertexts, computed on the GPU (requires m == Ng): d_pub is the
 * public matrix on the device (layout of sfft_keys_public), d_ct_out receives
 * count*2*F ciphertexts. The R bits are generated inside the kernel. */
int sfft_encrypt_bits_device(const sfft_params* p, const uint32_t* d_pub,
                             const double* h_re, const double* h_im, uint64_t count,
                             uint32_t F, uint32_t f, uint64_t enc_seed,
                             uint32_t* d_ct_out, void* stream);

/* GPU encryption of count arbitrary bits h_bits[c] in {0, 1} (EINVAL
 * otherwise) as ciphertext index c under enc_seed (the randomness layout of
 * sfft_encrypt_bits_device). Used for bootstrapping keys (sfft_key_bits). */
int sfft_encrypt_raw_bits_device(const sfft_params* p, const uint32_t* d_pub,
                                 const uint8_t* h_bits, uint64_t count, uint64_t enc_seed,
                                 uint32_t* d_ct_out, void* stream);

/* The bits a bootstrapping key encrypts (client side; sfft_refresh): h_bits[0]
 * = 1 (s_0 = 1), then bit b of s_j = -t_j mod q at 1 + (j - 1) ell + b, for
 * j = 1..n, b < ell. cap >= n ell + 1 bytes (EINVAL otherwise). */
int sfft_key_bits(const sfft_keys* k, uint8_t* h_bits, uint64_t cap);

/* Step 6, Dec (GSW'13; Lemma 2): x = <C'_{ell-1}, s> mod q, bit = [q/4 <= x
 * < 3q/4], words reassembled LSB first, value = signed word / 2^f.
 * h_rows points at row ell-1 of ciphertext 0; ciphertext j's row is
 * row_stride_words further on (row_stride_words = sfft_ct_words for a
 * packed ciphertext array, (n+1)*ell/32 for rows gathered by
 * sfft_gather_dec_rows). Writes count values to h_re / h_im (either may be
 * NULL) and the raw signed words to h_raw (NULL ok; 2*count entries,
 * re/im interleaved). Host only. */
int sfft_decrypt(const sfft_keys* k, const uint32_t* h_rows, uint64_t row_stride_words,
                 uint64_t count, uint32_t F, uint32_t f, double* h_re, double* h_im,
                 int64_t* h_raw);

/* Copies row ell-1 of each of n_ct device ciphertexts into d_rows (n_ct rows
 * of (n+1)*ell/32 words): what a client needs to decrypt. */
int sfft_gather_dec_rows(const sfft_params* p, const uint32_t* d_ct, uint64_t n_ct,
                         uint32_t* d_rows, void* stream);

/* ------------------------------------------------------------- circuits */

/* Smallest ell (multiple of 32, <= 8192) for which the static worst-case
 * noise bound of the FFT circuit stays below q/4 with m = Ng and error bound
 * chi (the leveled reading of the scheme's noise management; Sec. 5 ends by
 * pointing at refreshing). flags: the circuit variant (SFFT_PLAN_XCARRY or
 * SFFT_PLAN_NAND). 0 if none or if both variants are set. */
uint32_t sfft_min_ell(uint32_t N1, uint32_t N2, uint32_t F, uint32_t f, uint32_t n,
                      uint32_t chi, uint32_t flags);

typedef struct sfft_plan_info {
  uint64_t inputs, outputs;     /* ciphertexts in / out */
  uint64_t gates_and, gates_xor, gates_or, gates_not; /* logical gates after folding */
  uint64_t products;            /* ciphertext products (one per HA, AND, XOR, OR) */
  uint64_t levels;              /* multiplicative depth = launches of the plain evaluator */
  uint64_t max_level_width;     /* products in the widest level */
  uint64_t scratch_slots;       /* ciphertext slots of scratch needed by sfft_eval_fft */
  uint64_t scratch_bytes;
  uint64_t ct_words;
  uint32_t noise_bits;          /* bit length of the largest wire noise bound */
  uint32_t noise_ok;            /* bound < q/4 */
  uint32_t gate_kernel;         /* 1 integer-ALU kernel, 2 general tensor-core kernel,
                                   3 small-ciphertext tensor-core kernel (64 <= Ng <= 256) */
  uint32_t tc_columns;          /* tensor-core kernels: digit columns of a product row,
                                   (n+1) ceil(ell / dw) with dw = 11 bits (kernel 2) or
                                   8 bits (kernel 3); 0 otherwise */
  uint64_t gates_xadd;          /* linear exclusive-carry sums (SFFT_PLAN_XCARRY), no product */
} sfft_plan_info;

/* Builds the canonical gate circuit of a 1-D (N2 == 1) or row-column 2-D FFT
 * of F-bit words with f fraction bits (Sec. 4: bit reversal, butterflies of
 * fixed-point Wallace constant multipliers and ripple adders/subtractors;
 * Lemmas 3-9), levelises it (all products of one multiplicative depth form a
 * level) and uploads its gate descriptors to the device. Fails with EPARAM
 * if the static noise bound reaches q/4. flags: SFFT_PLAN_* below. */
#define SFFT_PLAN_ALLOW_NOISY 1u   /* build even if the noise bound fails */
#define SFFT_PLAN_INT_KERNEL 2u    /* integer-ALU gate kernel even where tensor cores apply */
/* The general tensor-core kernel (B operands expanded by a separate pass)
 * even where the small-ciphertext kernel applies (64 <= Ng <= 256); for
 * comparisons. EPARAM where the general kernel does not apply. */
#define SFFT_PLAN_TC_KERNEL 64u
/* Circuit variant (not the paper's): the full adder's carry is the sum of its
 * two half-adder carries, which are never both 1 (Lemma 6's OR, exact on
 * every input it meets), a linear gate (0, 1, 1, 0) with no ciphertext
 * product whose noise adds instead of growing by Ng. Fewer products and a
 * smaller ell (sfft_min_ell with the same flag); different ciphertexts. Linear
 * gates run after the products of their level. */
#define SFFT_PLAN_XCARRY 8u
/* Circuit variant (the paper's literal construction, Lemma 4 and Sec. 7's gate
 * counts): every gate that survives constant folding is built from GSW NAND
 * gates (1, 0, 0, -1), one ciphertext product each: NOT a = NAND(a, a), AND =
 * NOT(NAND), OR = NAND(NOT a, NOT b), a half adder t = NAND(a, b), XOR =
 * NAND(NAND(a, t), NAND(b, t)), AND = NAND(t, t). Several times the products
 * and a larger ell; decrypts to the same words. Exclusive with
 * SFFT_PLAN_XCARRY (EINVAL). */
#define SFFT_PLAN_NAND 16u
/* Variant (not the paper's, which multiplies by plaintext twiddles and notes
 * in Sec. 4 that a plaintext constant's bits show through the Wallace tree):
 * the FFT takes its twiddles as encrypted words and multiplies with the
 * encrypted-operand Wallace multiplier (every partial product an AND of two
 * ciphertexts). Inputs: the signal as without the flag, then one table of
 * M/2 complex words W_M^k = floor(cos(2 pi k / M) 2^f) + i floor(-sin(2 pi k /
 * M) 2^f), M = max(N1, N2), as samples N1 N2 + k (sfft_twiddles gives the
 * values; encrypt them with the signal in one sfft_encrypt_bits call).
 * Requires f <= F - 2 (W_M^0 = 2^f must fit a signed F-bit word). Same output
 * words as the plaintext-twiddle circuit. Combines with either gate variant. */
#define SFFT_PLAN_ENC_TWIDDLE 32u
int sfft_plan_create(const sfft_params* p, uint32_t N1, uint32_t N2, uint32_t F, uint32_t f,
                     uint32_t flags, sfft_plan** out);
int sfft_plan_info_get(const sfft_plan* plan, sfft_plan_info* info);
void sfft_plan_free(sfft_plan* plan);

/* Refresh (bootstrapping; Sec. 5 closes by pointing at refreshing, without a
 * construction): count ciphertexts are decrypted homomorphically under a
 * bootstrapping key, giving fresh-noise encryptions of the same bits. Row
 * ell - 1 of a ciphertext, c = (c_0..c_n), has phase x = <c, s> = sum_r K_r
 * sigma_r (mod q) with sigma_0 = 1, K_0 = c_0, and sigma_{j,b} = bit b of
 * s_j, K_{j,b} = c_j 2^b mod q. The circuit sums the top p = ceil(log2(n ell
 * + 1)) + 3 bits of every K_r (Lemma 8's Wallace stages, Lemma 7's ripple
 * adder, mod 2^p) and outputs [the top two bits of the sum differ]: the
 * decryption of c whenever its phase noise lies in [-q/8, q/4). Every term
 * is a bootstrapping-key ciphertext selected by a bit of c (a linear gate
 * beta C): the gate program is fixed, and each run patches the selected
 * gates' coefficients from the source ciphertexts on the device.
 * sfft_refresh_plan_create: inputs n ell + 1 (the bootstrapping key, i.e.
 * encryptions of sfft_key_bits), outputs count (EINVAL when count (n ell + 1)
 * p exceeds 2^28 / 7, the circuit's size bound); EPARAM if the output's static
 * noise bound reaches q/8 (it could not be refreshed again) unless
 * SFFT_PLAN_ALLOW_NOISY. flags: SFFT_PLAN_INT_KERNEL and the gate variants. */
int sfft_refresh_plan_create(const sfft_params* p, uint64_t count, uint32_t flags,
                             sfft_plan** out);
/* Smallest ell (multiple of 32, m = Ng) whose refresh output bound stays
 * below q/8; 0 if none up to 8192. */
uint32_t sfft_refresh_min_ell(uint32_t n, uint32_t chi, uint32_t flags);
/* d_bk: the n ell + 1 bootstrapping-key ciphertexts; d_src: the count
 * ciphertexts to refresh (only their rows ell - 1 are read); d_out: count
 * refreshed ciphertexts; scratch as sfft_eval_fft. One run at a time per plan
 * (the run rewrites the plan's gate coefficients). */
int sfft_refresh(sfft_plan* plan, const uint32_t* d_bk, const uint32_t* d_src, uint32_t* d_out,
                 uint32_t* d_scratch, uint64_t scratch_bytes, void* stream);

/* Word circuits: count independent operations on pairs of encrypted F-bit
 * two's-complement words (x, y), evaluated like an FFT plan (sfft_eval_fft and
 * sfft_eval_fft_host take any plan). Word k's x is input (2k) F + b, its y
 * input (2k + 1) F + b (the layout of sfft_encrypt_bits with re = x, im = y);
 * its result is output k F + b. Ops: (x + y) mod 2^F and (x - y) mod 2^F
 * (Sec. 4, Lemma 7), and the fixed-point product of two ciphertext words,
 * floor(x y / 2^f) mod 2^F, by the encrypted-operand Wallace multiplier
 * (partial products AND(x_ext[c - i], y_ext[i]) over T = f + F sign-extended
 * bits, Lemma 8's Wallace stages, Lemma 9's middle bits [f, f + F)). flags:
 * as sfft_plan_create (SFFT_PLAN_ENC_TWIDDLE has no effect). EINVAL unless
 * count >= 1 with count (f + F)^2 <= 2^28 (the circuit's size), 2 <= F <= 48,
 * f < F. */
#define SFFT_WORD_ADD 1u
#define SFFT_WORD_SUB 2u
#define SFFT_WORD_MUL 3u
int sfft_word_plan_create(const sfft_params* p, uint32_t op, uint64_t count, uint32_t F,
                          uint32_t f, uint32_t flags, sfft_plan** out);

/* Smallest ell of a word circuit (as sfft_min_ell; independent of count). */
uint32_t sfft_word_min_ell(uint32_t op, uint32_t F, uint32_t f, uint32_t n, uint32_t chi,
                           uint32_t flags);

/* Quantised twiddles W_M^k, k < M/2 (M a power of two >= 2): h_wr[k] =
 * floor(cos(2 pi k / M) 2^f), h_wi[k] = floor(-sin(2 pi k / M) 2^f), fp64
 * (Sec. 4's truncation read as floor). The client encrypts them for
 * SFFT_PLAN_ENC_TWIDDLE. h_wr, h_wi: M/2 entries each, caller-owned. */
int sfft_twiddles(uint32_t M, uint32_t f, int64_t* h_wr, int64_t* h_wi);

/* Step 4 on the server, plain level-by-level form: one kernel launch per
 * level, every product of the level evaluated in parallel. d_in holds
 * info.inputs ciphertexts, d_out receives info.outputs; d_scratch holds at
 * least info.scratch_bytes (caller-allocated, contents undefined on entry).
 * Device pointers must be 16-byte aligned. */
int sfft_eval_fft(sfft_plan* plan, const uint32_t* d_in, uint32_t* d_out,
                  uint32_t* d_scratch, uint64_t scratch_bytes, void* stream);

/* Waits for the stream and reports (then clears) the plan's device error
 * word: SFFT_ETIMEOUT if a bounded wait inside a gate kernel ran out since the
 * last check (the kernel then skipped its outputs and released its TMEM). */
int sfft_plan_check(sfft_plan* plan, void* stream);

/* Test hooks for parity at full size (the scope's sampled-gate check: gates
 * across all levels recomputed on a CPU from the GPU's own stored inputs).
 * sfft_eval_levels runs levels [l0, l1) of the plan's program (each level's
 * products, then its linear gates) on the caller's buffers, as sfft_eval_fft
 * does for the whole range, and the output fix-ups when l1 is the level
 * count; EINVAL unless l0 <= l1 <= levels. A level's gates read only slots
 * written by earlier levels and never write a slot the level reads, so a
 * caller may copy a gate's inputs out of the buffers before running its level
 * and its outputs after. sfft_plan_level returns level `level`'s gates in
 * launch order (products first, then linear gates; *n_products of them are
 * products): h_desc gets 4 words per gate (A, B, output 0, output 1), each
 * a reference with the region in bits 31..30 (0 scratch slot, 1 input, 2
 * output) and the ciphertext index in bits 29..0, 0xFFFFFFFF for an absent
 * output; ciphertext index x of a region starts at word x * sfft_ct_words of
 * its buffer. h_code gets code0 | code1 << 16 (each packs the signed nibbles
 * c0 | c1 << 4 | c2 << 8 | c3 << 12 of out = c0 P + c1 A + c2 B + c3
 * BitDecomp(A~) B, mod 2^ell), h_flags bit 0 = A~ is P - A (else A). With
 * every array NULL only the counts are written; otherwise cap must be at
 * least the level's gate count (EINVAL). */
int sfft_eval_levels(sfft_plan* plan, uint32_t l0, uint32_t l1, const uint32_t* d_in, uint32_t* d_out,
                     uint32_t* d_scratch, uint64_t scratch_bytes, void* stream);
int sfft_plan_level(const sfft_plan* plan, uint32_t level, uint32_t* h_desc, uint32_t* h_code,
                    uint8_t* h_flags, uint64_t cap, uint64_t* n_gates, uint64_t* n_products);

/* Same, end to end from host buffers: copies h_in to d_in, evaluates, copies
 * d_out to h_out and waits for the stream. Pinned host memory is fastest. */
int sfft_eval_fft_host(sfft_plan* plan, const uint32_t* h_in, uint32_t* h_out,
                       uint32_t* d_in, uint32_t* d_out, uint32_t* d_scratch,
                       uint64_t scratch_bytes, void* stream);

/* Host-only statistics of the compiled circuit (no device memory touched):
 * fills every field of sfft_plan_info as sfft_plan_create would with the
 * same flags (only SFFT_PLAN_XCARRY and SFFT_PLAN_NAND change the circuit). */
int sfft_circuit_info(const sfft_params* p, uint32_t N1, uint32_t N2, uint32_t F, uint32_t f,
                      uint32_t flags, sfft_plan_info* info);

/* Host-only plaintext run of the compiled device program (test hook): the
 * same levels, scratch slots, output fix-ups and adjusted gate coefficients
 * as the device evaluator, applied to bits (A~ = 1 - a when complemented;
 * out = c0 + c1 a + c2 b + c3 A~ b). h_in_bits: info.inputs bytes (0/1),
 * h_out_bits: info.outputs bytes. */
int sfft_program_eval_plain(const sfft_params* p, uint32_t N1, uint32_t N2, uint32_t F,
                            uint32_t f, uint32_t flags, const uint8_t* h_in_bits,
                            uint8_t* h_out_bits);

/* Host-only listing of the compiled device program of the FFT (N1 x N2
 * points, F-bit words with f fraction bits; Sec. 5's circuit, its gates
 * grouped into the levels that run in parallel, Sec. 7), gate by gate in
 * program order (level by level; no device memory touched). flags:
 * SFFT_PLAN_* as for sfft_plan_create; with SFFT_BATCH_PERSISTENT the circuit
 * is compiled as the persistent batch form compiles it (scratch slots reused
 * two levels after their last read) and dep_a / dep_b name the gates the
 * persistent launch waits for. Call with h_gates NULL for *count, then with
 * capacity >= *count. EPARAM: SFFT_BATCH_PERSISTENT with a circuit that has
 * linear gates. */
typedef struct sfft_gate_record {
  uint32_t a, b;          /* operands: region << 30 | slot (0 scratch, 1 inputs, 2 outputs) */
  uint32_t o0, o1;        /* outputs in the same form; 0xFFFFFFFF: none */
  uint32_t code;          /* nibbles c0..c3 of output 0 in bits 0..15, of output 1 in 16..31 */
  uint32_t flags;         /* bit 0: A complemented (A~ = P - A) */
  uint32_t level;         /* the gate's level, from 0 */
  uint32_t dep_a, dep_b;  /* gates that last wrote a / b before this level (0xFFFFFFFF: a
                             program input, or no persistent schedule was asked for) */
} sfft_gate_record;
int sfft_program_gates(const sfft_params* p, uint32_t N1, uint32_t N2, uint32_t F, uint32_t f,
                       uint32_t flags, sfft_gate_record* h_gates, uint64_t capacity,
                       uint64_t* count);

/* Host-only hooks of a refresh program: statistics, and a plaintext run with
 * key bits h_key_bits (n ell + 1 bytes) and the rows ell - 1 of the count
 * refreshed ciphertexts h_rows ((n + 1) ell / 32 words each), writing count
 * bits. */
int sfft_refresh_circuit_info(const sfft_params* p, uint64_t count, uint32_t flags,
                              sfft_plan_info* info);
int sfft_refresh_eval_plain(const sfft_params* p, uint64_t count, uint32_t flags,
                            const uint8_t* h_key_bits, const uint32_t* h_rows,
                            uint8_t* h_out_bits);

/* The same two host-only hooks for word circuits (sfft_word_plan_create). */
int sfft_word_circuit_info(const sfft_params* p, uint32_t op, uint64_t count, uint32_t F,
                           uint32_t f, uint32_t flags, sfft_plan_info* info);
int sfft_word_program_eval_plain(const sfft_params* p, uint32_t op, uint64_t count, uint32_t F,
                                 uint32_t f, uint32_t flags, const uint8_t* h_in_bits,
                                 uint8_t* h_out_bits);

/* sfft_eval_fft without any allocation (the paper has no counterpart; this
 * is a library service). For callers that must not call cudaMalloc while
 * evaluating -- e.g. a host application whose memory pool already reserved
 * the device memory, or a latency-critical serving loop that cannot afford
 * cudaMalloc's implicit device-wide synchronisation. The caller passes inputs
 * and outputs; intermediate ciphertexts live in a fixed array of
 * sfft_noalloc_scratch_bytes() (32 MiB) that the library reserves on every
 * GPU that loads it, held until the process exits. Plans whose
 * info.scratch_bytes exceed it are rejected with SFFT_EINVAL. The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture. All calls share the one
 * array, so calls that overlap on the GPU (other streams, other threads)
 * race; nothing in it needs clearing between calls (every slot is written
 * before it is read). Makes no cudaMalloc/cudaFree or allocating library
 * call. */
int sfft_eval_fft_noalloc(sfft_plan* plan, const uint32_t* d_in, uint32_t* d_out, void* stream);
uint64_t sfft_noalloc_scratch_bytes(void);

/* Kernel timing: when on, CUDA events are recorded on the launching stream
 * around every gate-kernel launch of sfft_eval_fft* (the tensor-core GEMM or
 * the integer kernel) and around every B expansion. sfft_plan_timing waits
 * for them and returns, since the last read, the summed gate-kernel and
 * expansion milliseconds, the number of levels launched and the products
 * they evaluated, then resets. Any output pointer may be NULL. */
int sfft_plan_set_timing(sfft_plan* plan, int on);
int sfft_plan_timing(sfft_plan* plan, double* gate_ms, double* expand_ms, uint64_t* launches,
                     uint64_t* products);

/* ------------------------------------------------------------- batches */

/* One encrypted-FFT request: 1-D (N2 == 1) or N1 x N2 2-D, F-bit words with
 * f fraction bits. */
typedef struct sfft_request {
  uint32_t N1, N2, F, f;
} sfft_request;

/* Batched form of step 4: the circuits of `count` requests are built and
 * their levels merged (level l of the batch = every request's products of
 * multiplicative depth l, evaluated by the same launches), so many requests
 * share each launch. GSW leveled evaluation has no evaluation key, so the
 * requests may come from different client key sets (same n, ell). Inputs and
 * outputs are the requests' ciphertexts concatenated in request order
 * (sfft_batch_offsets gives each request's first ciphertext). Unless
 * SFFT_BATCH_NO_GRAPH, sfft_batch_eval captures the whole launch sequence as
 * a CUDA graph on first use and replays it (two pointer sets are kept,
 * re-captured when a third appears or the stream changes; needs a non-default
 * stream). flags: SFFT_PLAN_* too. */
#define SFFT_BATCH_NO_GRAPH 4u
/* Persistent form: every product of the batch runs in ONE launch of the
 * small-ciphertext kernel (64 <= Ng <= 256; EPARAM otherwise, and for circuits with
 * linear gates such as SFFT_PLAN_XCARRY). Its CTAs claim gates in program
 * order; a gate starts once the gates that produced its two operands have
 * stored them and every gate two levels up is done (scratch slots are reused
 * two levels after their last read, so neighbouring levels overlap), and
 * publishes itself when its outputs are written. Every wait is bounded; one
 * that runs out stops the launch with SFFT_ETIMEOUT (sfft_batch_check).
 * Per evaluation one small launch restarts the claim counter and the level
 * counts first and the output fix-ups follow: three launches in all, graph-
 * replayed like the level-by-level form. Results are identical. */
#define SFFT_BATCH_PERSISTENT 128u
int sfft_batch_create(const sfft_params* p, const sfft_request* reqs, uint32_t count,
                      uint32_t flags, sfft_batch** out);
int sfft_batch_info_get(const sfft_batch* b, sfft_plan_info* info);
int sfft_batch_offsets(const sfft_batch* b, uint64_t* h_in_off, uint64_t* h_out_off);
int sfft_batch_eval(sfft_batch* b, const uint32_t* d_in, uint32_t* d_out, uint32_t* d_scratch,
                    uint64_t scratch_bytes, void* stream);
/* End to end from host buffers: H2D of all inputs, evaluation, D2H of all
 * outputs, then waits for the stream. */
int sfft_batch_eval_host(sfft_batch* b, const uint32_t* h_in, uint32_t* h_out, uint32_t* d_in,
                         uint32_t* d_out, uint32_t* d_scratch, uint64_t scratch_bytes,
                         void* stream);
/* End to end for count steps, double-buffered: step i copies h_in[i] into
 * d_in[i % 2] (on an internal copy stream, once step i - 2 has read that set),
 * evaluates into d_out[i % 2] on `stream` (a non-default stream), and copies
 * d_out[i % 2] to h_out[i] on a second copy stream while step i + 1 runs.
 * h_in / h_out: count pointers to host buffers (pinned for overlap; entries
 * may repeat), d_in / d_out: two device buffer sets each. Returns after every
 * copy has completed. */
int sfft_batch_eval_host_pipelined(sfft_batch* b, const uint32_t* const* h_in,
                                   uint32_t* const* h_out, uint32_t count,
                                   uint32_t* const* d_in, uint32_t* const* d_out,
                                   uint32_t* d_scratch, uint64_t scratch_bytes, void* stream);
int sfft_batch_check(sfft_batch* b, void* stream);
/* Test hook of the persistent form: sets its 32-bit run counter (the epoch
 * that readiness flags are compared with) and waits for the copy on stream.
 * Each run first advances the counter; at its wrap the flags are cleared and
 * the counter restarts at 1. EINVAL for a batch without SFFT_BATCH_PERSISTENT. */
int sfft_batch_set_epoch(sfft_batch* b, uint32_t epoch, void* stream);
/* Per-launch event timing (graph replay is bypassed while timing is on). */
int sfft_batch_set_timing(sfft_batch* b, int on);
int sfft_batch_timing(sfft_batch* b, double* gate_ms, double* expand_ms, uint64_t* launches,
                      uint64_t* products);
void sfft_batch_free(sfft_batch* b);

/* ------------------------------------------------------------- serving */

/* Continuous-batching server (north side of Fig. 1's step 4 under load).
 * A worker thread owns a stream and repeats a tick: admit queued requests
 * (FIFO) while the HBM budget has room for all their ciphertexts (scratch
 * wires, inputs, outputs) and fewer than max_active run, copying their input
 * ciphertexts in; then launch the next level of every active request
 * together; finished requests get their fix-ups and are copied out to the
 * client's h_out, and their memory is released once the copy completed. A
 * request arriving while others run joins at the next tick. hbm_budget_bytes
 * is allocated at creation (one arena) plus descriptor pools. All requests
 * share (n, ell); their client keys may differ. */
typedef struct sfft_server_stats {
  uint64_t completed, queued, active, ticks, tick_gates, peak_active;
  double p50_ms, p99_ms, max_ms;   /* submit-to-completion latency of completed requests */
} sfft_server_stats;

/* flags: SFFT_PLAN_XCARRY or SFFT_PLAN_NAND selects that circuit variant for
 * every request. */
int sfft_server_create(const sfft_params* p, uint64_t hbm_budget_bytes, uint32_t max_active,
                       uint32_t flags, sfft_server** out);
/* Queues one request. h_in: its input ciphertexts (layout of sfft_eval_fft's
 * d_in), h_out: room for its output ciphertexts; both caller-owned and valid
 * until sfft_server_wait returned for the ticket. ENOMEM if the request alone
 * exceeds the budget. */
int sfft_server_submit(sfft_server* sv, const sfft_request* req, const uint32_t* h_in,
                       uint32_t* h_out, uint64_t* ticket);
/* Compiles the circuit of a request shape (and uploads its device program)
 * ahead of its first submission, so that later submissions of this shape only
 * queue; submit compiles a new shape itself otherwise (seconds for large
 * circuits, outside the server's lock). Synchronous. */
int sfft_server_prepare(sfft_server* sv, const sfft_request* req);
/* Waits up to timeout_ms for the request (ETIMEOUT otherwise), reports its
 * submit-to-completion latency, and forgets the ticket. */
int sfft_server_wait(sfft_server* sv, uint64_t ticket, uint32_t timeout_ms, double* latency_ms);
int sfft_server_get_stats(sfft_server* sv, sfft_server_stats* st);
/* Stops the worker (queued requests are dropped, running ones finish). */
void sfft_server_free(sfft_server* sv);

/* Measured integer-pipe peak of the current GPU (the integer kernel's
 * roofline denominator): every SM at full occupancy runs 8 independent chains
 * per thread of one 32-bit operation, op 0 add.u32 (IADD3), 1 lop3.b32
 * (LOP3), 2 mad.lo.u32 (IMAD), 3 popc.b32 (POPC; each step also XORs the
 * count back, so two operations per counted step), `iters` x 32 steps per
 * chain (0: 4096); *ops_per_s = counted operations per second between CUDA
 * events on the legacy stream, best of two timed launches after one warm-up.
 * Allocates a small buffer; synchronises the device. */
int sfft_measure_int_peak(uint32_t op, uint32_t iters, double* ops_per_s);

/* Autotuner of the small-ciphertext tensor-core kernel (gate kernel 3, used
 * where 64 <= Ng <= 256): for each ring depth it can run (gates in flight per CTA,
 * 2 to 8 where shared memory allows) it times one level of n_gates half-adder
 * products of random ciphertexts at p with CUDA events on the legacy stream
 * (best of reps; 0 means 3), then keeps the fastest depth for the current
 * device and p's limb count: every later launch of the kernel there uses it.
 * h_us_per_gate (optional, 8 entries, index = depth - 1) receives the
 * microseconds per gate of each depth (0 where not run). Allocates and frees
 * its own buffers (4 n_gates ciphertexts) and synchronises the device.
 * EPARAM if the kernel does not take p; EINVAL unless 1 <= n_gates <= 2^24. */
int sfft_autotune_small(const sfft_params* p, uint64_t n_gates, uint32_t reps,
                        uint32_t* best_slots, double* h_us_per_gate);
/* Sets (nslots 2..8) or clears (0: the default of 4) the ring depth of the
 * small-ciphertext kernel for the current device and ell (32, 64, 96, 128). */
int sfft_small_kernel_set_slots(uint32_t ell, uint32_t nslots);

/* Evaluates a single level of gates given explicitly (test hook): gate g
 * computes, with A = d_a[g] (complemented to P - A first when
 * (flags[g] & 1)) and B = d_b[g],
 *   d_out0[g] = c0 P + c1 A + c2 B + c3 BitDecomp(A) B    (code0 = c0..c3)
 *   d_out1[g] likewise with code1 when flags[g] & 2.
 * d_a/d_b/d_out0/d_out1 are arrays of n_gates ciphertexts; codes are 4
 * signed nibbles c0 | c1 << 4 | c2 << 8 | c3 << 12 (two's complement).
 * kernel: 0 automatic, 1 integer ALU, 2 general tensor-core kernel, 3 small-
 * ciphertext tensor-core kernel (64 <= Ng <= 256); EPARAM if unsupported.
 * Synchronises the stream; SFFT_ETIMEOUT if a bounded device wait ran out. */
int sfft_gate_level(const sfft_params* p, const uint32_t* d_a, const uint32_t* d_b,
                    uint32_t* d_out0, uint32_t* d_out1, const uint16_t* h_code0,
                    const uint16_t* h_code1, const uint8_t* h_flags, uint64_t n_gates,
                    uint32_t kernel, void* stream);

/* Failure-detection test hook: the same level of gates on the tensor-core
 * kernel (EPARAM where it does not apply), except that every CTA's producer
 * withholds the B copy of K step `step`. That step's barrier never
 * completes, the kernel's bounded waits run out (about 2 s), every role
 * stops, the kernel drains its own MMAs, frees its tensor memory and
 * returns; the call then returns SFFT_ETIMEOUT and the context stays usable.
 * d_out0 is left undefined. */
int sfft_gate_level_withheld(const sfft_params* p, const uint32_t* d_a, const uint32_t* d_b,
                             uint32_t* d_out0, const uint16_t* h_code0, const uint8_t* h_flags,
                             uint64_t n_gates, uint32_t step, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SFFT_H */
