// Pipe-throughput microbenchmarks (perm_pipe_peaks in include/perm.h): the
// denominators of the roofline fractions the benchmark reports.  Each kernel
// runs 8 independent dependency chains per thread of one instruction kind on
// every SM and is timed with CUDA events; the chains are written out so the
// compiler keeps them.
#include <math.h>
#include <stdint.h>

#include "common.cuh"

namespace permgpu {

constexpr int kPeakIters = 256;   // outer iterations
constexpr int kPeakUnroll = 32;   // instructions per chain per iteration
constexpr int kPeakChains = 8;

template <int OP>
__global__ void __launch_bounds__(256) peak_kernel(unsigned long long* sink, uint32_t seed) {
  double d[kPeakChains];
  uint32_t u[kPeakChains];
  unsigned long long w[kPeakChains];
#pragma unroll
  for (int k = 0; k < kPeakChains; ++k) {
    d[k] = 1.0 + 1e-9 * (threadIdx.x + k);
    u[k] = seed * (threadIdx.x + 7u * k + 1u);
    w[k] = u[k];
  }
  const double b = 1.0 + 1e-12 * seed;
  const uint32_t bu = seed | 1u;
  for (int it = 0; it < kPeakIters; ++it) {
#pragma unroll
    for (int r = 0; r < kPeakUnroll; ++r) {
#pragma unroll
      for (int k = 0; k < kPeakChains; ++k) {
        if (OP == 0) asm volatile("fma.rn.f64 %0, %0, %1, %1;" : "+d"(d[k]) : "d"(b));
        if (OP == 1) asm volatile("add.rn.f64 %0, %0, %1;" : "+d"(d[k]) : "d"(b));
        if (OP == 2) asm volatile("mad.lo.u32 %0, %0, %1, %1;" : "+r"(u[k]) : "r"(bu));
        if (OP == 3) asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(w[k]) : "r"(u[k]), "r"(bu));
        if (OP == 4) asm volatile("shf.l.wrap.b32 %0, %0, %1, %0;" : "+r"(u[k]) : "r"(bu));
      }
    }
  }
  unsigned long long acc = 0;
#pragma unroll
  for (int k = 0; k < kPeakChains; ++k) acc += (unsigned long long)__double_as_longlong(d[k]) + u[k] + w[k];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

}  // namespace permgpu

using namespace permgpu;

extern "C" int perm_pipe_peaks(double* out, int count, void* stream) {
  if (!out || count < 1) return PERM_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PERM_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PERM_ECUDA;
  const int grid = sms * 4, block = 256;
  unsigned long long* sink = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&sink), sizeof(unsigned long long) * grid * block, s) != cudaSuccess) {
    cudaGetLastError();
    return PERM_ENOMEM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = PERM_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = PERM_ECUDA;
  void (*kernels[5])(unsigned long long*, uint32_t) = {peak_kernel<0>, peak_kernel<1>, peak_kernel<2>, peak_kernel<3>,
                                                       peak_kernel<4>};
  const double ops = (double)grid * block * kPeakIters * kPeakUnroll * kPeakChains;
  for (int k = 0; k < count; ++k) out[k] = NAN;  // written only after a successful timing
  for (int k = 0; k < 5 && k < count && rc == PERM_OK; ++k) {
    kernels[k]<<<grid, block, 0, s>>>(sink, 3u);  // warm-up
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      float ms = 0.f;
      if (cudaEventRecord(e0, s) != cudaSuccess) rc = PERM_ECUDA;
      if (!rc) kernels[k]<<<grid, block, 0, s>>>(sink, 3u + rep);
      if (!rc && cudaEventRecord(e1, s) != cudaSuccess) rc = PERM_ECUDA;
      if (!rc && cudaEventSynchronize(e1) != cudaSuccess) rc = PERM_ECUDA;
      if (!rc && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = PERM_ECUDA;
      if (rc) break;
      if (ms < best) best = ms;
    }
    if (!rc) out[k] = ops / (best * 1e-3);  // lane-instructions per second
  }
  if (cudaGetLastError() != cudaSuccess && rc == PERM_OK) rc = PERM_ECUDA;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(sink, s);
  if (cudaStreamSynchronize(s) != cudaSuccess && rc == PERM_OK) rc = PERM_ECUDA;
  return rc;
}
