// Pipe-throughput microbenchmarks (perm_pipe_peaks in include/perm.h): the
// denominators of the roofline fractions the benchmark reports.  Each kernel
// runs 8 independent dependency chains per thread of one instruction kind on
// every SM and is timed with CUDA events; the chains are written out so the
// compiler keeps them.
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
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return PERM_ECUDA;
  void (*kernels[5])(unsigned long long*, uint32_t) = {peak_kernel<0>, peak_kernel<1>, peak_kernel<2>, peak_kernel<3>,
                                                       peak_kernel<4>};
  int rc = PERM_OK;
  const double ops = (double)grid * block * kPeakIters * kPeakUnroll * kPeakChains;
  for (int k = 0; k < 5 && k < count; ++k) {
    kernels[k]<<<grid, block, 0, s>>>(sink, 3u);  // warm-up
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0, s);
      kernels[k]<<<grid, block, 0, s>>>(sink, 3u + rep);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        rc = PERM_ECUDA;
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) best = ms;
    }
    out[k] = ops / (best * 1e-3);  // lane-instructions per second
  }
  if (cudaGetLastError() != cudaSuccess) rc = PERM_ECUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(sink, s);
  cudaStreamSynchronize(s);
  return rc;
}
