// Measured integer-pipe peaks of the current GPU: the denominators of the
// integer kernel's roofline (32-bit limb additions and the logic, multiply
// and population-count operations around them).
//
// Each thread runs kChains independent dependency chains of one 32-bit
// operation (inline PTX, so that every step is the operation asked for and
// nothing folds), over enough warps to fill every SM; the rate is operations
// per second between two CUDA events around the launch. Chains are
// independent so that the pipe's throughput, not its latency, bounds the
// rate; the final values are stored so that no chain is dead.
#include <cuda_runtime.h>

#include <cstdint>

#include "common.h"
#include "plan.h"

namespace sfft {

namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 512;

template <int OP>
__global__ void __launch_bounds__(kPeakThreads) k_int_peak(uint32_t iters, uint32_t seed, uint32_t* sink) {
  uint32_t v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; c++) v[c] = seed + threadIdx.x * 131u + c * 7919u + blockIdx.x;
  const uint32_t k1 = seed | 1u, k2 = seed ^ 0x9E3779B9u;
  for (uint32_t it = 0; it < iters; it++) {
#pragma unroll
    for (int r = 0; r < 4; r++) {
#pragma unroll
      for (int c = 0; c < kChains; c++) {
        if (OP == 0)
          asm volatile("add.u32 %0, %0, %1;" : "+r"(v[c]) : "r"(k1));
        else if (OP == 1)
          asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(v[c]) : "r"(k1), "r"(k2));
        else if (OP == 2)
          asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(v[c]) : "r"(k1), "r"(k2));
        else
          asm volatile("{\n .reg .b32 t;\n popc.b32 t, %0;\n xor.b32 %0, %0, t;\n}\n" : "+r"(v[c]));
      }
    }
  }
  uint32_t acc = 0;
#pragma unroll
  for (int c = 0; c < kChains; c++) acc ^= v[c];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

}  // namespace

}  // namespace sfft

using namespace sfft;

extern "C" int sfft_measure_int_peak(uint32_t op, uint32_t iters, double* ops_per_s) {
  if (!ops_per_s || op > 3) return fail(SFFT_EINVAL, "op must be 0 (add), 1 (lop3), 2 (mad), 3 (popc)");
  if (iters == 0) iters = 4096;
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e, "device attributes");
  void* fn = op == 0 ? (void*)k_int_peak<0> : op == 1 ? (void*)k_int_peak<1> : op == 2 ? (void*)k_int_peak<2>
                                                                                  : (void*)k_int_peak<3>;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kPeakThreads, 0);
  if (e != cudaSuccess || per_sm < 1) per_sm = 1;
  const uint32_t blocks = (uint32_t)(sms * per_sm);
  uint32_t* sink = nullptr;
  e = cudaMalloc((void**)&sink, (size_t)blocks * kPeakThreads * 4);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 0;
  for (int rep = 0; rep < 3 && e == cudaSuccess; rep++) {   // the first launch warms up
    cudaEventRecord(e0, 0);
    switch (op) {
      case 0: k_int_peak<0><<<blocks, kPeakThreads>>>(iters, 12345u, sink); break;
      case 1: k_int_peak<1><<<blocks, kPeakThreads>>>(iters, 12345u, sink); break;
      case 2: k_int_peak<2><<<blocks, kPeakThreads>>>(iters, 12345u, sink); break;
      default: k_int_peak<3><<<blocks, kPeakThreads>>>(iters, 12345u, sink); break;
    }
    count_launches(1);
    cudaEventRecord(e1, 0);
    e = cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && (best == 0 || ms < best)) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (e != cudaSuccess) return cuda_fail(e, "integer peak kernel");
  // the popcount chain issues two operations per step (popc, xor); count popc only
  const double ops = (double)blocks * kPeakThreads * iters * 4.0 * kChains;
  *ops_per_s = best > 0 ? ops / (best / 1000.0) : 0;
  return SFFT_OK;
}
