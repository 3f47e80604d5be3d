// Dense real Ryser kernel (Alg. 1 in Nijenhuis-Wilf form, chunked as Alg. 3
// with the power-of-two chunks of Sec. 3.1.1), GB300-first:
//
//  * FP64 issues at 1/64 of the FP32 rate on this part, so the hot loop runs
//    on the integer pipes.  Every row of A is scaled by a power of two and
//    rounded once to 64-bit fixed point; the doubled row vector x' = 2x is then
//    an exact int64 per row (Y_i), updated by one int64 add per row and step
//    (no drift, unlike a binary64 running sum).
//  * Column n-1 is rounded to odd multiples and the other columns to even ones,
//    so Y_i is always odd and |Y_i| is (Y_i xor sign) | 1 - three integer ops.
//  * prod_i x_i carries a 62..63-bit mantissa in two 32-bit halves and a
//    power-of-two count: three 32x32->64 multiply-adds and one renormalising
//    shift per factor (relative error below 2^-60 per factor).
//  * Each step's signed term is split without rounding into a binary64 head
//    and a small tail, both assembled from the integer mantissa and exponent,
//    and added to a per-lane double-double with an exact Fast2Sum (Sec. 5's
//    "quad" outer sum, applied to every term): the only roundings left are
//    the 62-bit products and the double-double itself.
//  * The matrix is staged in shared memory as signed column increments
//    (+D_j and -D_j, j < n-1), column-contiguous; all lanes of a warp flip the
//    same column at the same step (aligned chunks, Sec. 3.1.1), so every
//    column read is a shared-memory broadcast.
//  * Lane partials are reduced warp -> CTA -> grid in a fixed order, so the
//    result is bitwise reproducible for a given n and launch shape.
#pragma once

#include "common.cuh"

namespace permgpu {

// Running product: mantissa M = (m1:m0) in [2^62, 2^63) (up to the initial
// value 2^62).  The renormalising shifts are accounted for by the caller.
struct Prod {
  uint32_t m0, m1;
};

__device__ __forceinline__ void prod_init(Prod& p) {
  p.m0 = 0u;
  p.m1 = 1u << 30;  // 2^62
}

// p <- p * A for A = a1:a0 < 2^63: v = M A / 2^64 rounded to nearest up to
// the dropped partial product m0*a0 (< 1 unit; +1/2 unit is added to the
// middle partial products, so products of integers that fit stay exact),
// then M <- v << (30 - pos) with pos the index of the top set bit of v_hi, so
// that M is back in [2^62, 2^63).  Returns pos (-1 if v_hi is zero, when the
// shift is 31).  The multiply-adds issue on the IMAD pipe and the shifts on the
// ALU pipe; the high limb of v comes from a carry-chained pair instead of a
// zero-extended 64-bit addend.  Intermediates stay below 2^64 because
// m1 < 2^31 and a1 < 2^31.
__device__ __forceinline__ uint32_t prod_mul(Prod& p, uint32_t a0, uint32_t a1) {
  uint32_t pos;
  asm("{\n\t"
      ".reg .u64 t, u;\n\t"
      ".reg .u32 ul, uh, vl, vh, s;\n\t"
      "mad.wide.u32 t, %2, %3, 2147483648;\n\t"
      "mad.wide.u32 u, %1, %4, t;\n\t"
      "mov.b64 {ul, uh}, u;\n\t"
      "mad.lo.cc.u32 vl, %2, %4, uh;\n\t"
      "madc.hi.u32 vh, %2, %4, 0;\n\t"
      "bfind.u32 %0, vh;\n\t"
      "sub.u32 s, 30, %0;\n\t"
      "shf.l.wrap.b32 %2, vl, vh, s;\n\t"
      "shl.b32 %1, vl, s;\n\t"
      "}"
      : "=r"(pos), "+r"(p.m0), "+r"(p.m1)
      : "r"(a0), "r"(a1));
  return pos;
}

// |Y| of an odd fixed-point row value Y (|Y| < 2^62) as (a0, a1), and the sign
// mask m (0 or all ones).
__device__ __forceinline__ void row_abs(unsigned long long Y, uint32_t& a0, uint32_t& a1, uint32_t& m) {
  uint32_t ylo = (uint32_t)Y;
  uint32_t yhi = (uint32_t)(Y >> 32);
  m = (uint32_t)((int32_t)yhi >> 31);
  a0 = (ylo ^ m) | 1u;
  a1 = yhi ^ m;
}

// The term sign * M * 2^(f+1-1023-62), M in [2^62, 2^63), as an unevaluated
// sum hi + lo of two binary64 numbers with no rounding: hi is M rounded to 53
// bits (the implicit bit placed on the exponent field f, the biased exponent
// minus one, clamped at 0 by the caller), lo = M - round(M) in [-512, 511]
// units of 2^(f+1-1023-62).  Both are assembled with integer operations; no
// FP64 instruction is used.
__device__ __forceinline__ void prod_to_dd(const Prod& p, uint32_t f, uint32_t signbit, double& hi, double& lo) {
  uint32_t rlo, rhi;
  asm("add.cc.u32 %0, %2, 512;\n\t"
      "addc.u32 %1, %3, 0;"
      : "=r"(rlo), "=r"(rhi)
      : "r"(p.m0), "r"(p.m1));
  const uint32_t lo32 = __funnelshift_r(rlo, rhi, 10);
  const uint32_t hi32 = (rhi >> 10) + (f << 20) + signbit;
  hi = __hiloint2double((int)hi32, (int)lo32);
  // remainder r = M - (R with its low 10 bits cleared), |r| <= 512; the tail
  // is (-1)^sign r 2^(f - 61 - 1023), assembled from integers as well: the
  // top bit of |r| sets the exponent, its (at most nine) lower bits the
  // fraction; tails below the normal range flush to zero
  const int32_t r = (int32_t)(p.m0 - (rlo & 0xFFFFFC00u));
  const uint32_t nr = (uint32_t)(r >> 31);
  const uint32_t mag = ((uint32_t)r ^ nr) - nr;
  const int lz = __clz((int)(mag | 1u));
  const int be = (int)f - 61 + 31 - lz;
  const uint32_t hw = ((nr & 0x80000000u) ^ signbit) | ((uint32_t)be << 20) | (((mag << lz) << 1) >> 12);
  lo = (mag == 0u || be <= 0) ? 0.0 : __hiloint2double((int)hw, 0);
}

// Shared-memory layout (dynamic): Dpm[(2j + s) * NP + i] for j < n-1,
// s = 0 (+D_ij, the column enters) or 1 (-D_ij, it leaves); then base[NP]
// (Y at g = 0), then NP zeros (the "update" of a chunk's first step).
template <int N>
struct RealLayout {
  static constexpr int NP = (N + 1) & ~1;  // rows padded to even: 16-byte pairs
  static constexpr int NCOL = N > 1 ? N - 1 : 0;
  static constexpr size_t kD = 0;
  static constexpr size_t kBase = kD + sizeof(long long) * 2 * NCOL * NP;
  static constexpr size_t kZero = kBase + sizeof(long long) * NP;  // NP zeros
  static constexpr size_t kBytes = kZero + sizeof(long long) * NP;
};

struct RealShared {
  int sum_s;       // sum of the row scale exponents s_i, plus the column scales
  int bound_log2;  // sum of k_i - 1 (row i's absolute sum in [2^(k_i-1), 2^k_i)) minus the column scales
  int nonfinite;
  int zero_row;
  int cexp[64];    // column scales (exact column equilibration)
};

// Stage A into shared memory as fixed-point column increments.
//   s_i = 61 - k_i with sum_j |a_ij| in [2^(k_i - 1), 2^k_i);
//   Q_ij = 2 round(a_ij 2^(s_i - 1)) for j < n-1 (even),
//   Q_{i,n-1} = 2 floor(a 2^(s_i - 1)) + 1 (odd);
//   Y_i(g) = sum_j delta_j Q_ij  (delta_j = +1 if column j is in the subset
//   or j = n-1, else -1)  represents x'_i = 2 x_i scaled by 2^s_i, and
//   |Y_i| <= sum_j |Q_ij| < 2^61 + n.
template <int N>
__device__ __forceinline__ void real_stage(const double* __restrict__ A, unsigned char* smem, RealShared& sh,
                                           bool equilibrate) {
  using L = RealLayout<N>;
  long long* D = reinterpret_cast<long long*>(smem + L::kD);
  long long* base = reinterpret_cast<long long*>(smem + L::kBase);
  long long* zero = reinterpret_cast<long long*>(smem + L::kZero);
  const int csum = column_scales<1>(A, N, sh.cexp, equilibrate);
  if (threadIdx.x == 0) {
    sh.sum_s = csum;
    sh.bound_log2 = -csum;
    sh.nonfinite = 0;
    sh.zero_row = 0;
  }
  __syncthreads();
  int i = threadIdx.x;
  if (i < N) {
    const double* row = A + (size_t)i * N;
    double absum = 0.0;
    int fin = 1;
    for (int j = 0; j < N; ++j) {
      double a = row[j];
      fin &= isfinite(a) ? 1 : 0;
      absum += ldexp(fabs(a), sh.cexp[j]);
    }
    int k = 0;
    if (fin && absum > 0.0) frexp(absum, &k);
    int s = 61 - k;
    long long qsum = 0;
    for (int j = 0; j < N - 1; ++j) {
      long long q = fin ? __double2ll_rn(ldexp(row[j], s - 1 + sh.cexp[j])) : 0;
      long long Q = 2 * q;
      qsum += Q;
      D[(2 * j) * L::NP + i] = 2 * Q;
      D[(2 * j + 1) * L::NP + i] = -2 * Q;
    }
    long long qn = fin ? 2 * __double2ll_rd(ldexp(row[N - 1], s - 1 + sh.cexp[N - 1])) + 1 : 1;
    base[i] = qn - qsum;
    zero[i] = 0;
    atomicAdd(&sh.sum_s, s);
    atomicAdd(&sh.bound_log2, k - 1);
    if (!fin) atomicOr(&sh.nonfinite, 1);
    if (fin && absum == 0.0) atomicOr(&sh.zero_row, 1);
  } else if (i < L::NP) {
    for (int j = 0; j < N - 1; ++j) {
      D[(2 * j) * L::NP + i] = 0;
      D[(2 * j + 1) * L::NP + i] = 0;
    }
    base[i] = 1;
    zero[i] = 0;
  }
  __syncthreads();
}

// From n = 32 on, the sweep walks Gray steps in pairs (four product chains,
// one CTA of 256 threads per SM); below, one step at a time with two chains
// and two CTAs per SM (measured: the pairs are 4 % faster at n = 32, 10 % at
// n = 40 and 48, and 1 - 14 % slower below 32; from n = 60 on the four chains
// would spill).  Chunks then have at least 2^7 steps (c >= ceil(log2 n) + 2).
template <int N>
constexpr bool kRealStepPairs = N >= 32 && N <= 59;

template <int N>
__global__ void __launch_bounds__(kBlock, (kRealStepPairs<N> ? 1 : 2)) ryser_real_kernel(RyserArgs a) {
  using L = RealLayout<N>;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ RealShared sh;
  real_stage<N>(static_cast<const double*>(a.A), smem, sh, a.mode == 0);
  const long long* D = reinterpret_cast<const long long*>(smem + L::kD);
  const long long* base = reinterpret_cast<const long long*>(smem + L::kBase);
  const long long* zero = reinterpret_cast<const long long*>(smem + L::kZero);

  // exponent bookkeeping, see prod_to_dd: the term is
  // sign * M * 2^(64N + 3 - sum_s - sum_lz - 62) in units of prod_i x_i.
  const int K1 = 64 * N + 1025 - sh.sum_s;
  const bool bad = sh.nonfinite || sh.bound_log2 + N > 1000;
  const bool skip = bad || sh.zero_row;

  dd acc = {0.0, 0.0};
  const int lane = threadIdx.x & 31;
  const uint64_t t_start = global_ns();
  const uint64_t warp_id = (uint64_t)(blockIdx.x * kBlock + threadIdx.x) >> 5;
  const uint64_t nwarps = (uint64_t)(gridDim.x * kBlock) >> 5;
  const uint64_t ngroups = skip ? 0 : (a.nchunks + 31) / 32;
  const uint32_t nsteps = 1u << a.c;

  for (uint64_t q = warp_id; q < ngroups; q += nwarps) {
    if (should_stop(a.abort_word, a.budget_ns, t_start, a.aborted)) break;
    const uint64_t kk = q * 32 + lane;
    const bool active = kk < a.nchunks;
    const uint64_t k = a.k_begin + kk;
    const uint64_t g0 = k << a.c;
    uint32_t tlo, tcnt;
    chunk_window(a, g0, active, tlo, tcnt);
    const uint32_t kb = (uint32_t)(k & 1u) << a.c;  // bit c of g, for the chunk's middle step
    const uint32_t gpar = (uint32_t)(g0 & 1u);      // parity of g0 (odd only when c = 0)

    // Y at Gray(g0): base plus every column whose Gray bit is set.  Bits below
    // c-1 of Gray(k 2^c) are zero.
    unsigned long long Y[N];
#pragma unroll
    for (int i = 0; i < N; ++i) Y[i] = (unsigned long long)base[i];
    const uint64_t G = gray64(g0);
    for (int j = (a.c > 0 ? a.c - 1 : 0); j < N - 1; ++j) {
      const long long msk = -(long long)((G >> j) & 1u);
      const long long* col = D + (size_t)(2 * j) * L::NP;
#pragma unroll
      for (int i = 0; i < N; ++i) Y[i] += (unsigned long long)(col[i] & msk);
    }

    if constexpr (kRealStepPairs<N>) {
      // Steps in pairs (t even, t + 1): the odd step always flips column 0
      // (ctz(t + 1) = 0), so every row is updated twice in a row and feeds four
      // independent product chains (even / odd rows of both steps).  Twice
      // the instruction-level parallelism per warp at the same work per step;
      // the chains need the registers of one CTA per SM.  2^c >= 2 here.
      for (uint32_t t = 0; t < nsteps; t += 2) {
        const int j = __ffs(t) - 1;
        const uint32_t sb = ((t | kb) >> (j + 1)) & 1u;
        const uint32_t sb1 = (((t + 1) | kb) >> 1) & 1u;  // column 0 at step t + 1
        const longlong2* col = reinterpret_cast<const longlong2*>(t ? D + (size_t)(2 * j + sb) * L::NP : zero);
        const longlong2* col0 = reinterpret_cast<const longlong2*>(D + (size_t)sb1 * L::NP);
        Prod pa, pb, pc, pd;
        prod_init(pa);
        prod_init(pb);
        prod_init(pc);
        prod_init(pd);
        uint32_t neg = 0, epos = 0, neg1 = 0, epos1 = 0;
#pragma unroll
        for (int p = 0; p < L::NP / 2; ++p) {
          const longlong2 d = col[p];
          const longlong2 e = col0[p];
          uint32_t a0, a1, ma, c0, c1, mc;
          Y[2 * p] += (unsigned long long)d.x;
          row_abs(Y[2 * p], a0, a1, ma);
          Y[2 * p] += (unsigned long long)e.x;
          row_abs(Y[2 * p], c0, c1, mc);
          epos += prod_mul(pa, a0, a1);
          epos1 += prod_mul(pc, c0, c1);
          neg += ma;
          neg1 += mc;
          if (2 * p + 1 < N) {
            uint32_t b0, b1, mb, e0, e1, me;
            Y[2 * p + 1] += (unsigned long long)d.y;
            row_abs(Y[2 * p + 1], b0, b1, mb);
            Y[2 * p + 1] += (unsigned long long)e.y;
            row_abs(Y[2 * p + 1], e0, e1, me);
            epos += prod_mul(pb, b0, b1);
            epos1 += prod_mul(pd, e0, e1);
            neg += mb;
            neg1 += me;
          }
        }
        epos += prod_mul(pa, pb.m0, pb.m1);
        epos1 += prod_mul(pc, pd.m0, pd.m1);
        double th, tl;
        int f = K1 - (30 * (N + 1) - (int)epos) - (N + 1);
        prod_to_dd(pa, (uint32_t)max(f, 0), (neg ^ t ^ gpar) << 31, th, tl);
        bool in = t - tlo < tcnt;
        dd_acc(acc, in ? th : 0.0, in ? tl : 0.0);
        f = K1 - (30 * (N + 1) - (int)epos1) - (N + 1);
        prod_to_dd(pc, (uint32_t)max(f, 0), (neg1 ^ (t + 1) ^ gpar) << 31, th, tl);
        in = t + 1 - tlo < tcnt;
        dd_acc(acc, in ? th : 0.0, in ? tl : 0.0);
      }
      acc = dd_make(acc.hi, acc.lo);  // renormalise the lane partial
      continue;
    }
    for (uint32_t t = 0; t < nsteps; ++t) {
      // column j = ctz(t) enters or leaves (Alg. 1: j = log2(Gray_t xor
      // Gray_{t-1}), entering iff bit j+1 of g is clear); t = 0 is the chunk's
      // start state and updates nothing (its column pointer reads zeros).
      const int j = __ffs(t) - 1;
      const uint32_t sb = ((t | kb) >> (j + 1)) & 1u;
      const longlong2* col = reinterpret_cast<const longlong2*>(t ? D + (size_t)(2 * j + sb) * L::NP : zero);
      Prod pa, pb;
      prod_init(pa);
      prod_init(pb);
      uint32_t neg = 0, epos = 0;  // -(number of negative factors), sum of pos
#pragma unroll
      for (int p = 0; p < L::NP / 2; ++p) {
        const longlong2 d = col[p];
        uint32_t a0, a1, ma, b0, b1, mb = 0, qb = 0;
        Y[2 * p] += (unsigned long long)d.x;
        row_abs(Y[2 * p], a0, a1, ma);
        if (2 * p + 1 < N) {
          Y[2 * p + 1] += (unsigned long long)d.y;
          row_abs(Y[2 * p + 1], b0, b1, mb);
        }
        const uint32_t qa = prod_mul(pa, a0, a1);
        if (2 * p + 1 < N) qb = prod_mul(pb, b0, b1);
        neg = neg + ma + mb;
        epos = epos + qa + qb;
      }
      epos += prod_mul(pa, pb.m0, pb.m1);
      // the N + 1 multiplies (N rows and the merge) shifted by sum(30 - pos)
      const int shifts = 30 * (N + 1) - (int)epos;
      const int f = K1 - shifts - (N + 1);
      const uint32_t signbit = (neg ^ t ^ gpar) << 31;
      double th, tl;
      prod_to_dd(pa, (uint32_t)max(f, 0), signbit, th, tl);
      const bool in = t - tlo < tcnt;
      dd_acc(acc, in ? th : 0.0, in ? tl : 0.0);
    }
    acc = dd_make(acc.hi, acc.lo);  // renormalise the lane partial
  }

  dd blk = dd_block_sum(acc);
  dd* part = static_cast<dd*>(a.part);
  if (threadIdx.x == 0) part[blockIdx.x] = blk;
  if (!arrive_last(a.counter)) return;
  if (threadIdx.x < 32) {
    dd tot = dd_sum_partials(part, gridDim.x);
    if (threadIdx.x == 0) {
      double* out = static_cast<double*>(a.out);
      int32_t st = PERM_OK;
      if (sh.nonfinite) st = PERM_EINVAL;
      else if (sh.bound_log2 + N > 1000) st = PERM_ERANGE;
      else if (*a.aborted) st = stop_status(*a.aborted);
      if (a.mode == 0) {
        const double f = (N & 1) ? 2.0 : -2.0;  // 4 (n mod 2) - 2
        out[0] = st != PERM_OK ? __longlong_as_double(0x7ff8000000000000ll)
                 : (sh.zero_row ? 0.0 : (tot.hi + tot.lo) * f);
      } else {
        out[0] = st != PERM_OK ? __longlong_as_double(0x7ff8000000000000ll) : tot.hi;
        out[1] = st != PERM_OK ? 0.0 : tot.lo;
      }
      if (a.status) *a.status = st;
      *a.counter = 0u;
    }
  }
}

}  // namespace permgpu
