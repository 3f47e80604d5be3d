// Shared device helpers of the permanent kernels (GB300, sm_103a).
//
// Nothing here is specific to one element type: double-double accumulation
// (the "quad as two doubles" outer sum of Sec. 5, with exact Fast2Sum / TwoSum
// steps), warp and block reductions in a fixed order, the launch argument
// block, cancellation, and the integer helpers of the fixed-point product.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "perm.h"

namespace permgpu {

constexpr int kBlock = 256;  // threads per CTA for every Ryser kernel
constexpr int kWarps = kBlock / 32;

// ----------------------------------------------------------- double-double

struct dd {
  double hi, lo;
};

__device__ __forceinline__ dd dd_make(double s, double e) {
  double h = s + e;
  dd r;
  r.lo = e - (h - s);
  r.hi = h;
  return r;
}

__device__ __forceinline__ dd dd_add(dd a, dd b) {
  double s = a.hi + b.hi;
  double bv = s - a.hi;
  double e = (a.hi - (s - bv)) + (b.hi - bv);
  e += a.lo + b.lo;
  return dd_make(s, e);
}

__device__ __forceinline__ dd dd_add_d(dd a, double b) {
  double s = a.hi + b;
  double bv = s - a.hi;
  double e = (a.hi - (s - bv)) + (b - bv);
  e += a.lo;
  return dd_make(s, e);
}

// acc += hi + lo.  The heads are added exactly with Dekker's Fast2Sum after
// ordering them by magnitude; for finite binary64 values the order of |x| is
// the unsigned order of the bit patterns without the sign, so the ordering is
// an integer compare and two selects.  That is three FP64 operations instead
// of Knuth's six (the FP64 pipe is the 1/64-rate unit here); the tails and
// the heads' rounding error are carried in acc.lo.
__device__ __forceinline__ void dd_acc(dd& acc, double hi, double lo) {
  const unsigned long long ua = (unsigned long long)__double_as_longlong(acc.hi) & 0x7FFFFFFFFFFFFFFFull;
  const unsigned long long ub = (unsigned long long)__double_as_longlong(hi) & 0x7FFFFFFFFFFFFFFFull;
  const bool sw = ub > ua;
  const double a = sw ? hi : acc.hi, b = sw ? acc.hi : hi;
  const double s = a + b;
  const double err = b - (s - a);
  acc.hi = s;
  acc.lo += err + lo;
}

__device__ __forceinline__ dd dd_shfl_down(dd v, int off) {
  dd r;
  r.hi = __shfl_down_sync(0xffffffffu, v.hi, off);
  r.lo = __shfl_down_sync(0xffffffffu, v.lo, off);
  return r;
}

// Fixed-order warp reduction (lane 0 holds the result).
__device__ __forceinline__ dd dd_warp_sum(dd v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = dd_add(v, dd_shfl_down(v, off));
  return v;
}

// ------------------------------------------------------------ launch block

// Arguments of one Ryser launch.  The chunk grid: chunk k covers steps
// g in [k 2^c, (k+1) 2^c); chunks [k_begin, k_begin + nchunks) are visited and
// only steps inside [g_begin, g_end) are accumulated.
struct RyserArgs {
  const void* A;      // element type given by the kernel
  int n;
  int c;              // log2 of the chunk length, 0..30
  int mode;           // 0: write the finished permanent, 1: write the raw range sum
  uint64_t g_begin, g_end;
  uint64_t k_begin, nchunks;
  void* part;         // per-CTA partials (scratch, gridDim.x entries)
  unsigned int* counter;  // arrival counter (scratch, zero before launch)
  void* out;
  int32_t* status;    // optional device status word
  const volatile uint32_t* abort_word;  // device view of a host-mapped word, or null
  unsigned int* aborted;                // scratch word next to the counter (zeroed)
  uint64_t budget_ns;                   // time budget of the sweep (perm_set_time_budget), 0: none
};

// Nanoseconds of the GPU's global timer.
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Cancellation and the time budget, checked between chunk groups: lane 0 reads
// the host-mapped abort word (perm_set_abort_word) and the time since t0 (the
// warp's start) once per group, and the warp follows it.  A warp that stops
// marks the launch (bit 0: aborted, bit 1: out of time) so that the finishing
// CTA reports PERM_EABORTED or PERM_ETIMEOUT.  Nothing waits.
__device__ __forceinline__ bool should_stop(const volatile uint32_t* word, uint64_t budget_ns, uint64_t t0,
                                            unsigned int* flag) {
  if (!word && !budget_ns) return false;
  uint32_t v = 0u;
  if ((threadIdx.x & 31) == 0) {
    if (word && *word != 0u) v = 1u;
    else if (budget_ns && global_ns() - t0 > budget_ns) v = 2u;
  }
  v = __shfl_sync(0xffffffffu, v, 0);
  if (v == 0u) return false;
  if ((threadIdx.x & 31) == 0) atomicOr(flag, v);
  return true;
}

// The status of a stopped launch from its flag word (0 if it ran to the end).
__device__ __forceinline__ int32_t stop_status(unsigned int flag) {
  return (flag & 1u) ? PERM_EABORTED : (flag & 2u) ? PERM_ETIMEOUT : PERM_OK;
}

// ------------------------------------------------ exact column equilibration

// Columns whose largest |entry| (complex: the larger part) lies more than a
// factor 2^kColGap below the largest column's are scaled by the power of two
// 2^c_j that brings them level with it; perm(A diag(2^c)) = perm(A) 2^(sum c),
// so the sum is taken back out of the result's exponent (exact).  Two reasons:
//  * the rows are rounded to a fixed point relative to their absolute sums, so
//    without the scale the entries of a column far below the others keep few
//    bits (or none);
//  * a column far above the others dominates every row sum x_i, the terms of
//    the sweep are then far larger than the permanent and cancel (with one
//    column 2^7 above the rest, n = 14 loses 20 bits to cancellation);
//    balanced columns avoid that.
// Matrices whose column maxima lie within a factor 2 of each other (random
// dense, Haar and the sparse workloads) keep c_j = 0: they are staged exactly
// as without equilibration.
constexpr int kColGap = 1;

// Only a sweep over all 2^(n-1) steps is equilibrated: the scale changes the
// individual terms (only their full sum scales by 2^(sum c)), so range sums
// (perm_range, perm_sparse_range, mode 1) stage the matrix unscaled and keep
// the terms of Alg. 1.
//
// W = 1: real entries A[i n + j]; W = 2: (re, im) pairs.  Threads j < n each
// scan one column (`rows`: one row, for a sweep whose toggles are the rows of
// A; perm(diag(2^c) A) = 2^(sum c) perm(A) as well); c[j] receives the
// exponent shift (0 everywhere unless `apply`).  Returns sum_j c_j (the same
// in every thread).  Contains __syncthreads().
template <int W>
__device__ __forceinline__ int column_scales(const double* __restrict__ A, int n, int* c, bool apply,
                                             bool rows = false) {
  __shared__ int s_emax, s_csum;
  if (threadIdx.x == 0) {
    s_emax = -100000;
    s_csum = 0;
  }
  __syncthreads();
  int e = -100000;  // a zero (or non-finite) column: no scale
  const int j = threadIdx.x;
  if (j < n) {
    double m = 0.0;
    for (int i = 0; i < n; ++i)
      for (int w = 0; w < W; ++w) m = fmax(m, fabs(A[((rows ? (size_t)j * n + i : (size_t)i * n + j)) * W + w]));
    if (m > 0.0 && isfinite(m)) {
      frexp(m, &e);
      atomicMax(&s_emax, e);
    }
  }
  __syncthreads();
  if (j < n) {
    const int cj = (apply && e > -100000 && s_emax - e > kColGap) ? s_emax - e : 0;
    c[j] = cj;
    if (cj) atomicAdd(&s_csum, cj);
  }
  __syncthreads();
  return s_csum;
}

// Gray code of step g (Sec. 2): bit j set <=> column j is in the subset.
__device__ __forceinline__ uint64_t gray64(uint64_t g) { return g ^ (g >> 1); }

// Step window of chunk k inside [g_begin, g_end): local t in [tlo, tlo + tcnt).
__device__ __forceinline__ void chunk_window(const RyserArgs& a, uint64_t g0, bool active, uint32_t& tlo,
                                             uint32_t& tcnt) {
  uint64_t len = 1ull << a.c;
  uint64_t lo = a.g_begin > g0 ? a.g_begin - g0 : 0;
  uint64_t hi = a.g_end > g0 ? a.g_end - g0 : 0;
  if (hi > len) hi = len;
  tlo = (uint32_t)lo;
  tcnt = (active && hi > lo) ? (uint32_t)(hi - lo) : 0u;
}

// Arrival protocol of the last CTA: every CTA stores its partial, the last one
// to arrive reads them all in index order.  Returns true in the last CTA.
__device__ __forceinline__ bool arrive_last(unsigned int* counter) {
  __shared__ unsigned int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned int prev = atomicAdd(counter, 1u);
    s_last = (prev == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0;
}

// Block-wide dd reduction (fixed order); result valid in thread 0.
__device__ __forceinline__ dd dd_block_sum(dd v) {
  __shared__ dd s_w[kWarps];
  v = dd_warp_sum(v);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) s_w[w] = v;
  __syncthreads();
  dd r = {0.0, 0.0};
  if (w == 0) {
    r = lane < kWarps ? s_w[lane] : dd{0.0, 0.0};
    r = dd_warp_sum(r);
  }
  __syncthreads();
  return r;
}

// Fixed-order sum of count dd partials by warp 0 (lane-strided, then tree).
__device__ __forceinline__ dd dd_sum_partials(const dd* p, int count) {
  dd r = {0.0, 0.0};
  int lane = threadIdx.x & 31;
  for (int i = lane; i < count; i += 32) r = dd_add(r, p[i]);
  return dd_warp_sum(r);
}

}  // namespace permgpu
