// Device-resident form of a compiled program and the launch helpers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "common.h"
#include "kargs.h"
#include "netlist.h"

namespace sfft {

struct DeviceProgram {
  GateDesc* desc = nullptr;
  GateAux* aux = nullptr;
  FixDesc* fix = nullptr;
  uint64_t n_fix = 0;
  PatchDesc* patch = nullptr;    // refresh programs: code patches applied before each run
  uint64_t n_patch = 0;
  std::vector<uint64_t> level_off;
  std::vector<uint64_t> lin_start;   // per level: first linear gate (after its products)
  uint64_t scratch_slots = 0;
  int* err = nullptr;            // device error word of the kernels
  uint32_t kernel = 0;           // KERNEL_AUTO / KERNEL_INT / KERNEL_TC / KERNEL_SM
  uint64_t max_width = 0;        // products in the widest level
  bool tc = false;               // levels run on the tensor-core kernel
  uint64_t scratch_bytes = 0;    // wire slots + expanded B operands
  uint64_t bx_off = 0;           // offset of the expanded B operands in scratch
  int device = -1;               // CUDA device that holds the program (current at creation)
};

// Reads and clears the device error word (synchronises the stream).
int check_device_error(int* err, cudaStream_t st);

int cuda_fail(cudaError_t e, const char* what);
int upload(const void* h, size_t bytes, void** d);
KArgs make_args(const Shape& s);
int launch_gates(const KArgs& a, cudaStream_t st);
// Linear gates (no ciphertext product) of one level.
int launch_linear(const KArgs& a, cudaStream_t st);
// Output fix-ups (copies, complements, constants) of n entries.
int launch_fixups(const FixDesc* d_fix, uint64_t n, const KArgs& a, cudaStream_t st);
// Process-wide count of this library's kernel launches (sfft_launch_count).
void count_launches(uint64_t n);
// Tensor-core gate kernel (tc.cu): shapes it supports, and its launcher.
bool tc_supported(const KArgs& a);
// Small-ciphertext tensor-core kernel (tc_small.cu): shapes it supports (Ng
// <= 256), its digit columns, its launcher (nslots 0: tuned or default ring
// depth) and the tuned ring depth per limb count on the current device.
bool sm_supported(const KArgs& a);
uint32_t sm_digit_columns(const KArgs& a);
int launch_gates_sm(const KArgs& a, cudaStream_t st);
int launch_gates_sm_slots(const KArgs& a, uint32_t nslots, cudaStream_t st);
int sm_set_tuned_slots(uint32_t L, uint32_t nslots);
// The gate kernel launch_gates runs for these arguments (a.kernel, the shape
// and a.bx_shared): KERNEL_SM, KERNEL_TC or KERNEL_INT; 0 when the kernel
// a.kernel forces does not support the shape.
uint32_t gate_kernel_for(const KArgs& a);
// Gate kernel a plan or batch requests from its flags (SFFT_PLAN_INT_KERNEL,
// SFFT_PLAN_TC_KERNEL, else automatic).
uint32_t plan_kernel(uint32_t flags);
// Digit columns of the tensor-core kernel that runs (0 for the integer kernel).
uint32_t gate_digit_columns(const KArgs& a);
int launch_gates_tc(const KArgs& a, cudaStream_t st);
// Failure-detection test: the same launch with K step `step`'s B copy withheld.
int launch_gates_tc_withheld(const KArgs& a, uint32_t step, cudaStream_t st);
// Bytes of the expanded B operand of one gate (0 if the shape is unsupported),
// and of the expansion buffer a launch of `gates` gates needs (levels run in
// L2-sized chunks of gates that share one buffer).
uint64_t tc_bx_bytes_per_gate(const KArgs& a);
uint64_t tc_bx_bytes(const KArgs& a, uint64_t gates);
// Digit columns of one row of the tensor-core product (elements x digits per
// element), 0 if the tensor-core kernel does not support the shape.
uint32_t tc_digit_columns(const KArgs& a);
// Scratch layout of a program: wire slots first, then (tensor-core kernel) the
// expanded B operands of the widest level, 256-byte aligned.
uint64_t scratch_layout(const Shape& s, uint64_t slots, uint64_t max_width, bool tc, uint64_t* bx_off);
int make_device_program(const Program& p, DeviceProgram* dp);
void free_device_program(DeviceProgram* dp);
// Optional per-launch CUDA-event timing of gate kernels.
// Event pairs around kernel launches, by kind: the gate kernels (the GEMM of
// the tensor-core path or the integer kernel) and the B expansion.
constexpr int kTimeGate = 0, kTimeExpand = 1;
struct Timer {
  bool on = false;
  std::vector<cudaEvent_t> pool[2];
  size_t used[2] = {0, 0};
  uint64_t launches = 0, products = 0;
  double last_expand_ms = 0;   // expansion time of the last drain
  cudaEvent_t next(int kind);   // an event from the kind's pool (grows on demand)
  double drain_ms();            // waits, sums the pairs, resets; returns the gate time
  ~Timer();
};

int run_program(const Shape& s, const DeviceProgram& dp, const uint32_t* d_in, uint32_t* d_out,
                uint32_t* d_scratch, uint64_t scratch_bytes, cudaStream_t st, Timer* tm = nullptr);
// Levels [l0, l1) of a program (the output fix-ups too when l1 is the last).
int run_levels(const Shape& s, const DeviceProgram& dp, uint32_t l0, uint32_t l1, const uint32_t* d_in,
               uint32_t* d_out, uint32_t* d_scratch, uint64_t scratch_bytes, cudaStream_t st,
               Timer* tm = nullptr);

}  // namespace sfft

// A compiled FFT plan (opaque in the C ABI).
struct sfft_plan {
  sfft::Shape s;
  sfft::Circuit circuit;
  sfft::Program prog;
  sfft::DeviceProgram dev;
  sfft::Timer timer;
  sfft::CircuitSpec spec;        // what the plan evaluates (FFT or word operations)
};
