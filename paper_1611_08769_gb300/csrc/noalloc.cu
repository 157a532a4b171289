// FFT evaluation that allocates nothing: the scratch pool is a fixed array in
// device global memory that this library reserves once, at module load.
//
// Who needs it: callers that must not call cudaMalloc during evaluation --
// for example a host application whose memory pool has already reserved the
// device memory (a fresh cudaMalloc would fail or fragment that pool), or a
// latency-critical serving loop where cudaMalloc's implicit device-wide
// synchronisation would stall work on other streams. They still pass their
// own input and output ciphertext buffers; only the intermediate wires live
// in the fixed array.
//
// The array is kNoAllocScratchBytes (32 MiB) on every GPU that loads the
// library, held until the process exits. Plans needing more scratch than that
// are rejected with SFFT_EINVAL.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "plan.h"

namespace {

constexpr uint64_t kNoAllocScratchBytes = 32ull << 20;
constexpr int kMaxDevices = 64;

// One array per device, shared by every call of sfft_eval_fft_noalloc.
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocScratchBytes / 4];

std::mutex g_mu;
uint32_t* g_scratch_ptr[kMaxDevices] = {};

// Device address of the array on the current device. Host code cannot use
// the symbol itself (it names a host-side stand-in), so the address is
// looked up once per device with that device current.
int scratch_on_current_device(uint32_t** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return sfft::cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return sfft::fail(SFFT_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return sfft::cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
    g_scratch_ptr[dev] = static_cast<uint32_t*>(p);
  }
  *out = g_scratch_ptr[dev];
  return SFFT_OK;
}

}  // namespace

extern "C" int sfft_eval_fft_noalloc(sfft_plan* pl, const uint32_t* d_in, uint32_t* d_out,
                                     void* stream) {
  if (!pl) return sfft::fail(SFFT_EINVAL, "plan is NULL");
  if (pl->dev.n_patch) return sfft::fail(SFFT_EINVAL, "a refresh plan runs through sfft_refresh");
  const uint64_t need = pl->dev.scratch_bytes;
  if (need > kNoAllocScratchBytes)
    return sfft::fail(SFFT_EINVAL, "plan needs " + std::to_string(need) +
                                       " bytes of scratch; sfft_eval_fft_noalloc holds at most " +
                                       std::to_string(kNoAllocScratchBytes) +
                                       " (use sfft_eval_fft with a caller buffer)");
  uint32_t* scratch = nullptr;
  int rc = scratch_on_current_device(&scratch);
  if (rc) return rc;
  // Every scratch slot is written by its producing gate before any gate reads
  // it, so nothing has to be cleared between calls.
  return sfft::run_program(pl->s, pl->dev, d_in, d_out, scratch, kNoAllocScratchBytes,
                           (cudaStream_t)stream, nullptr);
}

extern "C" uint64_t sfft_noalloc_scratch_bytes(void) { return kNoAllocScratchBytes; }
