// Launch arguments of the level kernels (shared by host launchers and kernels).
#pragma once

#include <cstdint>

#include "common.h"

namespace sfft {

// Producers of a gate's two operands (persistent launch; 0xFFFFFFFF: an input).
struct GateDeps {
  uint32_t a, b;
};

struct KArgs {
  const GateDesc* desc;
  const GateAux* aux;
  uint64_t n;            // gates in this launch
  uint32_t* base[4];     // region bases (region 3 = generated R for operand A)
  uint64_t gen_state;    // domain key of the generated R matrices
  uint32_t Ng, W, L, ell;
  uint64_t ctw;
  int* err;              // device error word (bounded waits that ran out), may be null
  uint32_t kernel;       // KERNEL_AUTO / KERNEL_INT / KERNEL_TC / KERNEL_SM
  uint8_t* bx;           // tensor-core kernel: expanded B operands (scratch)
  uint32_t bx_shared;    // 1: every gate has the same B operand (expanded once)
  void* timer;           // host: the Timer recording this launch's kernels, or null
  // Persistent launch across levels (small-ciphertext kernel, batches): gates
  // are claimed in program order from *claim; gate g waits until its
  // operands' producers are done (gflag[dep] >= *epoch; dep 0xFFFFFFFF: a
  // program input) and every gate of level glev[g] - 2 is done (ldone[l] >=
  // lwidth[l]; the counts and the claim are reset before each run), then
  // publishes gflag[g] = *epoch and counts itself in ldone[glev[g]] once its
  // outputs are stored. Null glev: one level per launch.
  const uint32_t* glev;
  const GateDeps* gdep;
  const uint32_t* lwidth;
  unsigned long long* ldone;
  uint32_t* gflag;
  uint32_t* claim;
  const uint32_t* epoch;
};

// KERNEL_TC: the general tensor-core kernel (B expanded by a separate pass);
// KERNEL_SM: the small-ciphertext tensor-core kernel (64 <= Ng <= 256, whole gates
// per CTA, B converted in the kernel).
constexpr uint32_t KERNEL_AUTO = 0, KERNEL_INT = 1, KERNEL_TC = 2, KERNEL_SM = 3;

// Error codes written to KArgs::err by kernels.
constexpr int KERR_MMA_TIMEOUT = 1;

}  // namespace sfft
