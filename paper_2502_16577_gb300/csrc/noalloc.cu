// perm_f64_noalloc: the dense real permanent without any allocation.
//
// perm() takes its scratch (one double-double partial per CTA and an arrival
// counter) from cudaMallocAsync on the caller's stream.  Some callers cannot
// call the CUDA allocator at all: code running under a framework that has
// reserved the device memory up front and forbids other allocations, hard
// real-time loops that allow no allocation after start-up, or hosts whose
// memory policy only permits allocation during initialisation.  This entry
// point serves them: its scratch is a fixed array in the library's own device
// memory (file-scope __device__ storage), so a call allocates nothing.
//
// The array is shared by every call on a device and keeps the last call's
// contents; the arrival counter is cleared by each call before its kernel.
// Two calls whose kernels overlap on the GPU (different streams, or calls
// from several host threads without ordering) race on it: order them.
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace permgpu {

// Enough for 4096 CTAs (16 bytes each) plus the counter: far above the
// resident grid of one GB300 (152 SMs x 2 CTAs).
constexpr size_t kNoAllocScratchBytes = 64 * 1024 + 256;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct NoAllocDevice {
  void* scratch = nullptr;  // device address of g_noalloc_scratch
};

// Per-device set-up, once, with that device current: the device address of
// the scratch array (its host-side name is only a stand-in and must never be
// passed to a kernel).
static int noalloc_device(NoAllocDevice& out) {
  static std::mutex mu;
  static NoAllocDevice cache[kNoAllocMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return PERM_ECUDA;
  std::lock_guard<std::mutex> lock(mu);
  NoAllocDevice& d = cache[dev];
  if (!d.scratch) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
      cudaGetLastError();
      return PERM_ECUDA;
    }
    d.scratch = ptr;
  }
  out = d;
  return PERM_OK;
}

__global__ void noalloc_trivial_kernel(double* out, int32_t* status) {
  if (threadIdx.x == 0) {
    out[0] = 1.0;
    if (status) *status = PERM_OK;
  }
}

}  // namespace permgpu

using namespace permgpu;

extern "C" int perm_f64_noalloc(const double* A, int n, double* out, int32_t* status, void* stream) {
  if (n < 0 || n > PERM_NMAX) return PERM_ERANGE;
  if (!out || (n > 0 && !A)) return PERM_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  NoAllocDevice nd;
  int rc = noalloc_device(nd);
  if (rc) return rc;
  if (n == 0) {
    noalloc_trivial_kernel<<<1, 32, 0, s>>>(out, status);
    return cudaGetLastError() == cudaSuccess ? PERM_OK : PERM_ECUDA;
  }
  KernelEntry ke = n <= 24 ? real_entry_lo(n) : n <= 44 ? real_entry_mid(n) : real_entry_hi(n);
  if (!ke.fn) return PERM_EINVAL;
  const uint64_t N = 1ull << (n - 1);
  RyserLaunch L;  // the launch shape of perm() for this matrix
  rc = plan_ryser_launch(ke, n, 0, N, L);
  if (rc) return rc;
  const int grid = L.grid, c = L.c;
  const uint64_t nchunks = L.nchunks;
  // the fixed array must hold one partial per CTA and the counter
  const size_t part_bytes = sizeof(dd) * (size_t)grid;
  if (part_bytes + 2 * sizeof(unsigned int) > kNoAllocScratchBytes) return PERM_ENOMEM;
  unsigned int* counter = reinterpret_cast<unsigned int*>(static_cast<char*>(nd.scratch) + part_bytes);
  if (cudaMemsetAsync(counter, 0, 2 * sizeof(unsigned int), s) != cudaSuccess) return PERM_ECUDA;
  RyserArgs args;
  memset(&args, 0, sizeof(args));
  args.A = A;
  args.n = n;
  args.c = c;
  args.mode = 0;
  args.g_begin = 0;
  args.g_end = N;
  args.k_begin = 0;
  args.nchunks = nchunks;
  args.part = nd.scratch;
  args.counter = counter;
  args.out = out;
  args.status = status;
  args.abort_word = current_abort_word();
  args.aborted = counter + 1;
  args.budget_ns = current_time_budget();
  void* params[] = {&args};
  if (cudaLaunchKernel(ke.fn, dim3(grid), dim3(kBlock), params, ke.smem, s) != cudaSuccess) {
    cudaGetLastError();
    return PERM_ECUDA;
  }
  return PERM_OK;
}
