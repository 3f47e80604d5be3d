// Dense real Ryser kernel with extended-precision products: the "quad"
// inner-product variable of Sec. 5 (Table 3's QQ/DQ variants keep the
// product of the x_i in double-double).  Same Gray-code sweep, staging and
// exact fixed-point rows as ryser_real_kernel; what changes:
//
//  * Column n-1 is rounded like the others (the default kernel rounds it to
//    odd multiples, a perturbation of 2^-61 of the row sum that would
//    dominate here), so the rows are exact whenever every a_ij 2^(60-k_i) is
//    an integer (2^(k_i-1) <= sum_j |a_ij| < 2^k_i), as for inputs on a
//    2^-53 grid.  A row value may then be zero; a zero factor makes the
//    running mantissa zero, and such terms are dropped.
//  * prod_i x_i carries a 128-bit mantissa (two 64-bit words) per chain.
//    Each factor |Y_i| is first normalised to [2^63, 2^64), so one factor
//    costs one 64 x 128 -> top-128-bit product and a shift of at most two
//    bits; the relative error is below 2^-123 per factor (2^-61 in the
//    default kernel).
//  * Each term is split into a 53-bit head (truncated) and the rounded
//    remainder, assembled from the mantissa with integer operations and one
//    integer-to-binary64 conversion; the split loses at most 2^-105 of the
//    term.
//  * The per-lane double-double is renormalised after every step, so its low
//    word never grows beyond half an ulp of the high word.
//  * The permanent is returned unevaluated as (hi, lo).
#pragma once

#include "real.cuh"

namespace permgpu {

// Running product: M = h 2^64 + l in [2^126, 2^127), or zero after a zero
// factor (every later multiply keeps it zero).
struct XProd {
  unsigned long long h, l;
};

__device__ __forceinline__ void xprod_init(XProd& p) {
  p.h = 1ull << 62;
  p.l = 0ull;
}

// Shift a 128-bit value hi:lo left by s in [0, 63].
__device__ __forceinline__ void shl128(unsigned long long& hi, unsigned long long& lo, uint32_t s) {
  hi = (hi << s) | ((lo >> 1) >> (63 - s));
  lo <<= s;
}

// p <- floor(M A / 2^64) less under 3 units (dropped: l0 a0 and the low
// words of l1 a0 and l0 a1), then shifted left by s so that M is back in
// [2^126, 2^127); returns s.  With M in [2^126, 2^127) and A in [2^63, 2^64)
// the unshifted value lies in [2^125 - 3, 2^127), so s is 0, 1 or 2 (31 for
// a zero product).  PTX over 32-bit limbs: seven multiply-adds in one carry
// chain, column by column, and a funnel-shift renormalisation.
__device__ __forceinline__ uint32_t xprod_mul(XProd& p, unsigned long long A) {
  uint32_t s;
  asm("{\n\t"
      ".reg .u32 h0, h1, l0, l1, a0, a1, r0, r1, r2, r3, t;\n\t"
      "mov.b64 {h0, h1}, %1;\n\t"
      "mov.b64 {l0, l1}, %2;\n\t"
      "mov.b64 {a0, a1}, %3;\n\t"
      "mul.hi.u32 r0, l1, a0;\n\t"
      "mul.hi.u32 t, l0, a1;\n\t"
      "add.cc.u32 r0, r0, t;\n\t"
      "addc.u32 r1, 0, 0;\n\t"
      "mad.lo.cc.u32 r0, l1, a1, r0;\n\t"
      "madc.hi.cc.u32 r1, l1, a1, r1;\n\t"
      "addc.u32 r2, 0, 0;\n\t"
      "mad.lo.cc.u32 r0, h0, a0, r0;\n\t"
      "madc.hi.cc.u32 r1, h0, a0, r1;\n\t"
      "addc.u32 r2, r2, 0;\n\t"
      "mad.lo.cc.u32 r1, h0, a1, r1;\n\t"
      "madc.hi.cc.u32 r2, h0, a1, r2;\n\t"
      "addc.u32 r3, 0, 0;\n\t"
      "mad.lo.cc.u32 r1, h1, a0, r1;\n\t"
      "madc.hi.cc.u32 r2, h1, a0, r2;\n\t"
      "addc.u32 r3, r3, 0;\n\t"
      "mad.lo.cc.u32 r2, h1, a1, r2;\n\t"
      "madc.hi.u32 r3, h1, a1, r3;\n\t"
      "bfind.u32 t, r3;\n\t"
      "sub.u32 %0, 30, t;\n\t"
      "shf.l.wrap.b32 r3, r2, r3, %0;\n\t"
      "shf.l.wrap.b32 r2, r1, r2, %0;\n\t"
      "shf.l.wrap.b32 r1, r0, r1, %0;\n\t"
      "shl.b32 r0, r0, %0;\n\t"
      "mov.b64 %1, {r2, r3};\n\t"
      "mov.b64 %2, {r0, r1};\n\t"
      "}"
      : "=r"(s), "+l"(p.h), "+l"(p.l)
      : "l"(A));
  return s;
}

// Merge two chains: M <- top 128 bits of Ma Mb / 2^128, renormalised; returns
// the left shift (1..3: the unshifted value lies in [2^124 - 3, 2^126); 63
// when a chain is zero).
// Dropped: la*lb and the low words of the cross products (< 3 units).
__device__ __forceinline__ uint32_t xprod_merge(XProd& a, const XProd& b) {
  const unsigned long long hh_hi = __umul64hi(a.h, b.h);
  const unsigned long long hh_lo = a.h * b.h;
  const unsigned long long c1 = __umul64hi(a.h, b.l);
  const unsigned long long c2 = __umul64hi(a.l, b.h);
  unsigned long long lo = hh_lo + c1;
  unsigned long long hi = hh_hi + (lo < c1 ? 1ull : 0ull);
  lo += c2;
  hi += lo < c2 ? 1ull : 0ull;
  const uint32_t s = (uint32_t)__clzll((long long)hi) - 1u;
  shl128(hi, lo, s);
  a.h = hi;
  a.l = lo;
  return s;
}

// The term sign * M * 2^E as hi + lo, fb = E + 1149 the biased binary64
// exponent of hi (M's top word lies in [2^62, 2^63), or M is zero).  hi
// keeps the top 53 bits of M (truncated); lo is the remaining 74 bits,
// rounded to 53 bits by one conversion and moved to its exponent by an
// integer add.  Terms whose head is below the normal range are flushed to
// zero; tails below it too.
__device__ __forceinline__ void xprod_to_dd(const XProd& p, int fb, unsigned long long sign, double& hi,
                                            double& lo) {
  if (fb <= 0 || p.h == 0ull) {
    hi = 0.0;
    lo = 0.0;
    return;
  }
  const unsigned long long hb = ((unsigned long long)(fb - 1) << 52) + (p.h >> 10);
  hi = __longlong_as_double((long long)(hb | sign));
  const unsigned long long rem = ((p.h & 0x3FFull) << 54) | (p.l >> 10);
  const double r = __ull2double_rn(rem);  // exact zero only for rem == 0
  const long long rb = __double_as_longlong(r);
  const int ef = (int)(rb >> 52) + fb - 1139;  // exponent field of rem 2^(E+10)
  lo = (rem == 0ull || ef <= 0)
           ? 0.0
           : __longlong_as_double((long long)(((unsigned long long)rb + ((unsigned long long)(long long)(fb - 1139) << 52)) | sign));
}

// |Y| shifted left by lz = clz(|Y|) into [2^63, 2^64) (zero for Y = 0: the
// PTX shift is defined for a count of 64), and the sign mask m (0 or ~0).
__device__ __forceinline__ unsigned long long row_norm(unsigned long long Y, uint32_t& lz, uint32_t& m) {
  const unsigned long long sm = (unsigned long long)((long long)Y >> 63);
  const unsigned long long ay = (Y ^ sm) - sm;
  lz = (uint32_t)__clzll((long long)ay);
  m = (uint32_t)sm;
  unsigned long long r;
  asm("shl.b64 %0, %1, %2;" : "=l"(r) : "l"(ay), "r"(lz));
  return r;
}

// After real_stage: replace the odd rounding of column n-1 in base[i] by the
// round-to-nearest of the other columns.  Both use the row scale s_i of
// real_stage; base[i] holds Q_{i,n-1} - sum_{j<n-1} Q_ij.
template <int N>
__device__ __forceinline__ void realx_exact_last_column(const double* __restrict__ A, unsigned char* smem,
                                                        const RealShared& sh) {
  using L = RealLayout<N>;
  long long* base = reinterpret_cast<long long*>(smem + L::kBase);
  const int i = threadIdx.x;
  if (i < N && !sh.nonfinite) {
    const double* row = A + (size_t)i * N;
    double absum = 0.0;
    for (int j = 0; j < N; ++j) absum += ldexp(fabs(row[j]), sh.cexp[j]);  // as real_stage
    int k = 0;
    if (absum > 0.0) frexp(absum, &k);
    const double v = ldexp(row[N - 1], 61 - k - 1 + sh.cexp[N - 1]);
    base[i] += 2 * __double2ll_rn(v) - (2 * __double2ll_rd(v) + 1);
  }
  __syncthreads();
}

template <int N>
__global__ void __launch_bounds__(kBlock, (N <= 40 ? 2 : 1)) ryser_realx_kernel(RyserArgs a) {
  using L = RealLayout<N>;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ RealShared sh;
  real_stage<N>(static_cast<const double*>(a.A), smem, sh, a.mode == 0);
  realx_exact_last_column<N>(static_cast<const double*>(a.A), smem, sh);
  const long long* D = reinterpret_cast<const long long*>(smem + L::kD);
  const long long* base = reinterpret_cast<const long long*>(smem + L::kBase);
  const long long* zero = reinterpret_cast<const long long*>(smem + L::kZero);

  // Exponent bookkeeping.  Row i holds Y_i = 2 x_i 2^(s_i).  Chain factors
  // enter as |Y_i| 2^(lz_i) with lz_i = clz(|Y_i|); every multiply divides by
  // 2^64 and shifts left by its return value, the merge divides by 2^128.
  // With SH the sum of all lz_i and shifts, both chains starting at 2^126:
  //   M = 2^124 prod_i |Y_i| 2^(SH - 64 N),
  // so |prod_i x_i| = M 2^E with E = 64 N - 124 - SH - sum_s - N and the
  // biased exponent of the head is fb = E + 1149 = KX - SH.
  const int KX = 63 * N + 1025 - sh.sum_s;
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
    const uint32_t kb = (uint32_t)(k & 1u) << a.c;
    const uint32_t gpar = (uint32_t)(g0 & 1u);

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

    for (uint32_t t = 0; t < nsteps; ++t) {
      const int j = __ffs(t) - 1;
      const uint32_t sb = ((t | kb) >> (j + 1)) & 1u;
      const longlong2* col = reinterpret_cast<const longlong2*>(t ? D + (size_t)(2 * j + sb) * L::NP : zero);
      XProd pa, pb;
      xprod_init(pa);
      xprod_init(pb);
      uint32_t neg = 0, sh_sum = 0;
#pragma unroll
      for (int p = 0; p < L::NP / 2; ++p) {
        const longlong2 d = col[p];
        Y[2 * p] += (unsigned long long)d.x;
        {
          uint32_t lz, m;
          const unsigned long long A = row_norm(Y[2 * p], lz, m);
          sh_sum += lz + xprod_mul(pa, A);
          neg += m;
        }
        if (2 * p + 1 < N) {
          Y[2 * p + 1] += (unsigned long long)d.y;
          uint32_t lz, m;
          const unsigned long long A = row_norm(Y[2 * p + 1], lz, m);
          sh_sum += lz + xprod_mul(pb, A);
          neg += m;
        }
      }
      sh_sum += xprod_merge(pa, pb);
      const unsigned long long sign = (unsigned long long)((neg ^ t ^ gpar) & 1u) << 63;
      double th, tl;
      xprod_to_dd(pa, KX - (int)sh_sum, sign, th, tl);
      const bool in = t - tlo < tcnt;
      dd_acc(acc, in ? th : 0.0, in ? tl : 0.0);
      acc = dd_make(acc.hi, acc.lo);
    }
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
      const double nan = __longlong_as_double(0x7ff8000000000000ll);
      tot = dd_make(tot.hi, tot.lo);
      if (a.mode == 0) {
        const double f = (N & 1) ? 2.0 : -2.0;  // 4 (n mod 2) - 2, exact on both words
        out[0] = st != PERM_OK ? nan : (sh.zero_row ? 0.0 : tot.hi * f);
        out[1] = st != PERM_OK ? 0.0 : (sh.zero_row ? 0.0 : tot.lo * f);
      } else {
        out[0] = st != PERM_OK ? nan : tot.hi;
        out[1] = st != PERM_OK ? 0.0 : tot.lo;
      }
      if (a.status) *a.status = st;
      *a.counter = 0u;
    }
  }
}

}  // namespace permgpu
