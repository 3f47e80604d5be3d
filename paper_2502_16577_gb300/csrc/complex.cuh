// Dense complex Ryser kernel (Alg. 1 over complex entries, chunked as Alg. 3
// with power-of-two chunks, Sec. 3.1.1).
//
// Rows are scaled by a power of two per row (taken from sum_j |re| + |im|) and
// rounded once to 64-bit fixed point, so the doubled row vector x' = 2x is an
// exact pair of int64 per row.  The running product z = prod_i x'_i keeps a
// shared exponent for its real and imaginary parts, both held as signed
// 62-bit integers split into a signed high limb and a 31-bit low limb, so
// that every partial product is a signed 32x32->64 multiply-add with no sign
// handling:  (p1 2^31 + p0)(y1 2^31 + y0) = p1 y1 2^62 + (p1 y0 + p0 y1) 2^31 + ...
// After each complex multiply the pair is renormalised so that the larger part
// has its top bit at 2^60.  Each part of a term is split exactly into a
// binary64 head and tail and added to double-double lane partials with an
// exact two-sum (dd_acc, Sec. 5).
#pragma once

#include "common.cuh"
#include "real.cuh"

namespace permgpu {

struct CProd {
  int32_t r1, i1;    // signed high limbs (bits 31..62)
  uint32_t r0, i0;   // low 31-bit limbs
};

__device__ __forceinline__ void cprod_init(CProd& p) {
  p.r1 = 1 << 29;  // 2^60 (real part), imaginary part 0
  p.r0 = 0u;
  p.i1 = 0;
  p.i0 = 0u;
}

// p <- p * y for y = (yr, yi) signed with |yr|, |yi| < 2^61.  Returns the
// renormalising shift s (the product was multiplied by 2^(s-62)).
//   middle partial products (scale 2^31):
//     tr = r1 yr0 + r0 yr1 - i1 yi0 - i0 yi1,  ti = r1 yi0 + r0 yi1 + i1 yr0 + i0 yr1
//   high partial products (scale 2^62) plus the carried middle part:
//     vr = r1 yr1 - i1 yi1 + (tr >> 31),  vi = r1 yi1 + i1 yr1 + (ti >> 31)
//   then the larger part's top bit is shifted to 2^60 and both parts are
//   split back into limbs.  Written as PTX signed wide multiply-adds with the
//   negated limbs formed once: a quarter fewer instructions than the same
//   arithmetic in C++ (measured), with bitwise-identical results.
__device__ __forceinline__ int cprod_mul(CProd& p, long long yr, long long yi) {
  int s;
  asm("{\n\t"
      ".reg .s64 tr, ti, vr, vi;\n\t"
      ".reg .s32 yr1, yr0, yi1, yi0, ni1, ni0, vrh, vih, m1, m2, a1, a2, w, pos;\n\t"
      ".reg .u32 ul, uh;\n\t"
      "mov.b64 {ul, uh}, %5;\n\t"
      "shf.l.wrap.b32 yr1, ul, uh, 1;\n\t"
      "and.b32 yr0, ul, 0x7FFFFFFF;\n\t"
      "mov.b64 {ul, uh}, %6;\n\t"
      "shf.l.wrap.b32 yi1, ul, uh, 1;\n\t"
      "and.b32 yi0, ul, 0x7FFFFFFF;\n\t"
      "neg.s32 ni1, %3;\n\t"
      "neg.s32 ni0, %4;\n\t"
      "mul.wide.s32 tr, %1, yr0;\n\t"
      "mad.wide.s32 tr, %2, yr1, tr;\n\t"
      "mad.wide.s32 tr, ni1, yi0, tr;\n\t"
      "mad.wide.s32 tr, ni0, yi1, tr;\n\t"
      "mul.wide.s32 ti, %1, yi0;\n\t"
      "mad.wide.s32 ti, %2, yi1, ti;\n\t"
      "mad.wide.s32 ti, %3, yr0, ti;\n\t"
      "mad.wide.s32 ti, %4, yr1, ti;\n\t"
      "shr.s64 tr, tr, 31;\n\t"
      "shr.s64 ti, ti, 31;\n\t"
      "mad.wide.s32 vr, %1, yr1, tr;\n\t"
      "mad.wide.s32 vr, ni1, yi1, vr;\n\t"
      "mad.wide.s32 vi, %1, yi1, ti;\n\t"
      "mad.wide.s32 vi, %3, yr1, vi;\n\t"
      "mov.b64 {ul, vrh}, vr;\n\t"
      "mov.b64 {ul, vih}, vi;\n\t"
      "shr.s32 m1, vrh, 31;\n\t"
      "xor.b32 a1, vrh, m1;\n\t"
      "shr.s32 m2, vih, 31;\n\t"
      "xor.b32 a2, vih, m2;\n\t"
      "or.b32 w, a1, a2;\n\t"
      "bfind.u32 pos, w;\n\t"  // -1 when both parts are tiny: shift 29
      "sub.s32 %0, 28, pos;\n\t"
      "shl.b64 vr, vr, %0;\n\t"
      "shl.b64 vi, vi, %0;\n\t"
      "mov.b64 {ul, uh}, vr;\n\t"
      "shf.l.wrap.b32 %1, ul, uh, 1;\n\t"
      "and.b32 %2, ul, 0x7FFFFFFF;\n\t"
      "mov.b64 {ul, uh}, vi;\n\t"
      "shf.l.wrap.b32 %3, ul, uh, 1;\n\t"
      "and.b32 %4, ul, 0x7FFFFFFF;\n\t"
      "}"
      : "=r"(s), "+r"(p.r1), "+r"(p.r0), "+r"(p.i1), "+r"(p.i0)
      : "l"(yr), "l"(yi));
  return s;
}

template <int N>
struct CplxLayout {
  static constexpr int NCOL = N > 1 ? N - 1 : 0;
  // D[(2j + s) * N + i] as (re, im) longlong2, then base[N], then zero[N]
  static constexpr size_t kD = 0;
  static constexpr size_t kBase = kD + sizeof(longlong2) * 2 * NCOL * N;
  static constexpr size_t kZero = kBase + sizeof(longlong2) * N;
  static constexpr size_t kBytes = kZero + sizeof(longlong2) * N;
};

struct CplxShared {
  int sum_s;       // row scales plus column scales
  int bound_log2;  // sum of k_i - 1 minus the column scales
  int nonfinite;
  int zero_row;
  int cexp[64];    // column scales (exact column equilibration)
};

// Q_ij = round(a_ij 2^s_i) (both parts), s_i = 60 - k_i with
// sum_j |re| + |im| in [2^(k_i-1), 2^k_i): |Y_i| <= 2^60 per part.
template <int N>
__device__ __forceinline__ void cplx_stage(const double* __restrict__ A, unsigned char* smem, CplxShared& sh,
                                           bool equilibrate) {
  using Lo = CplxLayout<N>;
  longlong2* D = reinterpret_cast<longlong2*>(smem + Lo::kD);
  longlong2* base = reinterpret_cast<longlong2*>(smem + Lo::kBase);
  longlong2* zero = reinterpret_cast<longlong2*>(smem + Lo::kZero);
  const int csum = column_scales<2>(A, N, sh.cexp, equilibrate);
  if (threadIdx.x == 0) {
    sh.sum_s = csum;
    sh.bound_log2 = -csum;
    sh.nonfinite = 0;
    sh.zero_row = 0;
  }
  __syncthreads();
  int i = threadIdx.x;
  if (i < N) {
    const double* row = A + 2 * (size_t)i * N;
    double absum = 0.0;
    int fin = 1;
    for (int j = 0; j < 2 * N; ++j) {
      double v = row[j];
      fin &= isfinite(v) ? 1 : 0;
      absum += ldexp(fabs(v), sh.cexp[j >> 1]);
    }
    int k = 0;
    if (fin && absum > 0.0) frexp(absum, &k);
    const int s = 60 - k;
    long long sr = 0, si = 0;
    for (int j = 0; j < N - 1; ++j) {
      long long qr = fin ? __double2ll_rn(ldexp(row[2 * j], s + sh.cexp[j])) : 0;
      long long qi = fin ? __double2ll_rn(ldexp(row[2 * j + 1], s + sh.cexp[j])) : 0;
      sr += qr;
      si += qi;
      D[(2 * j) * N + i] = make_longlong2(2 * qr, 2 * qi);
      D[(2 * j + 1) * N + i] = make_longlong2(-2 * qr, -2 * qi);
    }
    long long nr = fin ? __double2ll_rn(ldexp(row[2 * (N - 1)], s + sh.cexp[N - 1])) : 0;
    long long ni = fin ? __double2ll_rn(ldexp(row[2 * (N - 1) + 1], s + sh.cexp[N - 1])) : 0;
    base[i] = make_longlong2(nr - sr, ni - si);
    zero[i] = make_longlong2(0, 0);
    atomicAdd(&sh.sum_s, s);
    atomicAdd(&sh.bound_log2, k - 1);
    if (!fin) atomicOr(&sh.nonfinite, 1);
    if (fin && absum == 0.0) atomicOr(&sh.zero_row, 1);
  }
  __syncthreads();
}

template <int N>
__global__ void __launch_bounds__(kBlock, (N <= 8 ? 2 : 1)) ryser_cplx_kernel(RyserArgs a) {
  using Lo = CplxLayout<N>;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ CplxShared sh;
  cplx_stage<N>(static_cast<const double*>(a.A), smem, sh, a.mode == 0);
  const longlong2* D = reinterpret_cast<const longlong2*>(smem + Lo::kD);
  const longlong2* base = reinterpret_cast<const longlong2*>(smem + Lo::kBase);
  const longlong2* zero = reinterpret_cast<const longlong2*>(smem + Lo::kZero);
  const bool bad = sh.nonfinite || sh.bound_log2 + N > 1000;
  const bool skip = bad || sh.zero_row;
  // Each chain starts at 2^60 (= 1) and every one of the N + 1 multiplies
  // (N rows, then the merge of the two chains) scales by 2^(s - 62), so
  // prod_i Y_i = z 2^(62 (N+1) - 120 - sum shifts), and with Y_i = 2 x_i 2^s_i
  // the term prod_i x_i = z 2^(ebase - sum shifts).
  const int ebase = 62 * (N + 1) - 120 - sh.sum_s - N;

  dd accr = {0.0, 0.0}, acci = {0.0, 0.0};
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

    long long Yr[N], Yi[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      Yr[i] = base[i].x;
      Yi[i] = base[i].y;
    }
    const uint64_t G = gray64(g0);
    for (int j = (a.c > 0 ? a.c - 1 : 0); j < N - 1; ++j) {
      const long long msk = -(long long)((G >> j) & 1u);
      const longlong2* col = D + (size_t)(2 * j) * N;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        Yr[i] += col[i].x & msk;
        Yi[i] += col[i].y & msk;
      }
    }

    for (uint32_t t = 0; t < nsteps; ++t) {
      const int j = __ffs(t) - 1;
      const uint32_t sb = ((t | kb) >> (j + 1)) & 1u;
      const longlong2* col = t ? D + (size_t)(2 * j + sb) * N : zero;
      CProd pa, pb;
      cprod_init(pa);
      cprod_init(pb);
      int sa = 0, sbb = 0;
#pragma unroll
      for (int i = 0; i < N; i += 2) {
        const longlong2 d0 = col[i];
        Yr[i] += d0.x;
        Yi[i] += d0.y;
        sa += cprod_mul(pa, Yr[i], Yi[i]);
        if (i + 1 < N) {
          const longlong2 d1 = col[i + 1];
          Yr[i + 1] += d1.x;
          Yi[i + 1] += d1.y;
          sbb += cprod_mul(pb, Yr[i + 1], Yi[i + 1]);
        }
      }
      // merge chain b into chain a: b = (pb.r1 2^31 + pb.r0, ...) < 2^61 per part
      const long long br_ = ((long long)pb.r1 << 31) | pb.r0;
      const long long bi_ = ((long long)pb.i1 << 31) | pb.i0;
      const int sm = cprod_mul(pa, br_, bi_);
      const long long zr = ((long long)pa.r1 << 31) | pa.r0;
      const long long zi = ((long long)pa.i1 << 31) | pa.i0;
      const int e = ebase - (sa + sbb + sm);
      // each part as an exact head + tail pair: head = round(z), tail = z - head
      // (|tail| <= 2^8), both scaled by 2^e (powers of two: exact)
      const double hr = (double)zr, hi_ = (double)zi;
      const double lr = (double)(zr - __double2ll_rn(hr)), li = (double)(zi - __double2ll_rn(hi_));
      const double sc = ldexp(((t ^ gpar) & 1u) ? -1.0 : 1.0, e);
      const bool in = t - tlo < tcnt;
      dd_acc(accr, in ? hr * sc : 0.0, in ? lr * sc : 0.0);
      dd_acc(acci, in ? hi_ * sc : 0.0, in ? li * sc : 0.0);
    }
    accr = dd_make(accr.hi, accr.lo);
    acci = dd_make(acci.hi, acci.lo);
  }

  dd blkr = dd_block_sum(accr);
  dd blki = dd_block_sum(acci);
  dd* part = static_cast<dd*>(a.part);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = blkr;
    part[2 * blockIdx.x + 1] = blki;
  }
  if (!arrive_last(a.counter)) return;
  if (threadIdx.x < 32) {
    dd tr = {0.0, 0.0}, ti = {0.0, 0.0};
    for (unsigned int b = threadIdx.x; b < gridDim.x; b += 32) {
      tr = dd_add(tr, part[2 * b]);
      ti = dd_add(ti, part[2 * b + 1]);
    }
    tr = dd_warp_sum(tr);
    ti = dd_warp_sum(ti);
    if (threadIdx.x == 0) {
      double* out = static_cast<double*>(a.out);
      int32_t st = PERM_OK;
      if (sh.nonfinite) st = PERM_EINVAL;
      else if (sh.bound_log2 + N > 1000) st = PERM_ERANGE;
      else if (*a.aborted) st = stop_status(*a.aborted);
      const double nan = __longlong_as_double(0x7ff8000000000000ll);
      if (a.mode == 0) {
        const double f = (N & 1) ? 2.0 : -2.0;
        out[0] = st != PERM_OK ? nan : (sh.zero_row ? 0.0 : (tr.hi + tr.lo) * f);
        out[1] = st != PERM_OK ? nan : (sh.zero_row ? 0.0 : (ti.hi + ti.lo) * f);
      } else {
        out[0] = st != PERM_OK ? nan : tr.hi;
        out[1] = st != PERM_OK ? 0.0 : tr.lo;
        out[2] = st != PERM_OK ? nan : ti.hi;
        out[3] = st != PERM_OK ? 0.0 : ti.lo;
      }
      if (a.status) *a.status = st;
      *a.counter = 0u;
    }
  }
}

// ------------------------------------------------------------------------
// Two lanes per chunk (n >= 16).  The single-lane kernel above holds all n
// complex rows of its chunk in registers (about 255 registers at n = 32, one
// CTA per SM).  Here lane pair (2m, 2m+1) walks one chunk: each lane keeps
// half of the rows and one product chain, one shuffle and one complex
// multiply combine the halves, so twice as many warps stay resident for
// n + 2 instead of n + 1 complex multiplies per step.  Every term is computed
// by both lanes of the pair; the lane whose parity matches the step keeps it,
// and every second step both lanes split their kept term exactly into
// binary64 head + tail (integer assembly) and add it to their double-double
// partials.

struct CTerm {
  int32_t r1, i1;
  uint32_t r0, i0;
  int e;  // value = (r + i im) 2^e with r = r1 2^31 + r0
};

__device__ __forceinline__ CTerm cterm_mul(CTerm a, CTerm b) {
  CProd p;
  p.r1 = a.r1;
  p.i1 = a.i1;
  p.r0 = a.r0;
  p.i0 = a.i0;
  const long long br = ((long long)b.r1 << 31) | b.r0, bi = ((long long)b.i1 << 31) | b.i0;
  const int s = cprod_mul(p, br, bi);
  return CTerm{p.r1, p.i1, p.r0, p.i0, a.e + b.e + 62 - s};
}

// v 2^E (signed v, |v| < 2^62) as an exact head + tail (see prod_to_dd),
// negated when neg is set; zero for v = 0 or below the normal range.
__device__ __forceinline__ void cpart_to_dd(long long v, int E, uint32_t neg, double& h, double& l) {
  const unsigned long long sgn = (unsigned long long)(v >> 63);
  const unsigned long long mag = ((unsigned long long)v ^ sgn) - sgn;
  const int lz = __clzll((long long)(mag | 1ull));
  const unsigned long long nm = mag << (lz - 1);
  Prod p;
  p.m0 = (uint32_t)nm;
  p.m1 = (uint32_t)(nm >> 32);
  const int f = E - (lz - 1) + 62 + 1022;
  const uint32_t signbit = ((uint32_t)sgn ^ (0u - neg)) & 0x80000000u;
  prod_to_dd(p, (uint32_t)max(f, 0), signbit, h, l);
  if (mag == 0 || f < 1) h = l = 0.0;
}

template <int N>
__global__ void __launch_bounds__(kBlock, 2) ryser_cplx2_kernel(RyserArgs a) {
  constexpr int R = (N + 1) / 2;  // rows per lane
  using Lo = CplxLayout<N>;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ CplxShared sh;
  cplx_stage<N>(static_cast<const double*>(a.A), smem, sh, a.mode == 0);
  const longlong2* D = reinterpret_cast<const longlong2*>(smem + Lo::kD);
  const longlong2* base = reinterpret_cast<const longlong2*>(smem + Lo::kBase);
  const bool bad = sh.nonfinite || sh.bound_log2 + N > 1000;
  const bool skip = bad || sh.zero_row;
  // x_i = Y_i 2^(-s_i - 1).  The padded row of an odd n is 2^60 (a multiplier
  // of full precision for cprod_mul, which scales by 2^-62 and renormalises),
  // taken back out of the exponent here.
  const int eoff = -(sh.sum_s + N) - ((N & 1) ? 60 : 0);

  dd accr = {0.0, 0.0}, acci = {0.0, 0.0};
  const int lane = threadIdx.x & 31, li = lane & 1;
  const uint64_t t_start = global_ns();
  const uint64_t warp_id = (uint64_t)(blockIdx.x * kBlock + threadIdx.x) >> 5;
  const uint64_t nwarps = (uint64_t)(gridDim.x * kBlock) >> 5;
  const uint64_t ngroups = skip ? 0 : (a.nchunks + 15) / 16;  // 16 chunks per warp
  const uint32_t nsteps = 1u << a.c;

  for (uint64_t q = warp_id; q < ngroups; q += nwarps) {
    if (should_stop(a.abort_word, a.budget_ns, t_start, a.aborted)) break;
    const uint64_t kk = q * 16 + (lane >> 1);
    const bool active = kk < a.nchunks;
    const uint64_t k = a.k_begin + kk;
    const uint64_t g0 = k << a.c;
    uint32_t tlo, tcnt;
    chunk_window(a, g0, active, tlo, tcnt);
    const uint32_t kb = (uint32_t)(k & 1u) << a.c;
    const uint32_t gpar = (uint32_t)(g0 & 1u);

    long long Yr[R], Yi[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = li * R + r;
      const longlong2 b = i < N ? base[i] : make_longlong2(1ll << 60, 0);
      Yr[r] = b.x;
      Yi[r] = b.y;
    }
    const uint64_t G = gray64(g0);
    for (int j = (a.c > 0 ? a.c - 1 : 0); j < N - 1; ++j) {
      const long long msk = -(long long)((G >> j) & 1u);
      const longlong2* col = D + (size_t)(2 * j) * N + li * R;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (li * R + r < N) {
          Yr[r] += col[r].x & msk;
          Yi[r] += col[r].y & msk;
        }
      }
    }

    CTerm keep = {0, 0, 0u, 0u, 0};
    uint32_t kneg = 0u;
    for (uint32_t t = 0; t < nsteps; ++t) {
      if (t) {
        const int j = __ffs(t) - 1;
        const uint32_t sb = ((t | kb) >> (j + 1)) & 1u;
        const longlong2* col = D + (size_t)(2 * j + sb) * N + li * R;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if (li * R + r < N) {
            const longlong2 d = col[r];
            Yr[r] += d.x;
            Yi[r] += d.y;
          }
        }
      }
      CProd p;
      cprod_init(p);
      int ssum = 0;
#pragma unroll
      for (int r = 0; r < R; ++r) ssum += cprod_mul(p, Yr[r], Yi[r]);
      CTerm v{p.r1, p.i1, p.r0, p.i0, -60 + 62 * R - ssum};
      const CTerm o{__shfl_xor_sync(0xffffffffu, v.r1, 1), __shfl_xor_sync(0xffffffffu, v.i1, 1),
                    __shfl_xor_sync(0xffffffffu, v.r0, 1), __shfl_xor_sync(0xffffffffu, v.i0, 1),
                    __shfl_xor_sync(0xffffffffu, v.e, 1)};
      v = cterm_mul(li ? o : v, li ? v : o);  // both lanes: (lane 0 half) x (lane 1 half)
      if ((t & 1u) == (uint32_t)li) {
        keep = v;
        kneg = (t ^ gpar) & 1u;
      }
      if ((t & 1u) || t + 1 == nsteps) {
        const uint32_t tk = (t & ~1u) + (uint32_t)li;  // the step this lane kept
        const bool in = tk <= t && tk - tlo < tcnt;
        const long long zr = ((long long)keep.r1 << 31) | keep.r0;
        const long long zi = ((long long)keep.i1 << 31) | keep.i0;
        double hr, lr, hi_, li_;
        cpart_to_dd(zr, keep.e + eoff, kneg, hr, lr);
        cpart_to_dd(zi, keep.e + eoff, kneg, hi_, li_);
        dd_acc(accr, in ? hr : 0.0, in ? lr : 0.0);
        dd_acc(acci, in ? hi_ : 0.0, in ? li_ : 0.0);
      }
    }
    accr = dd_make(accr.hi, accr.lo);
    acci = dd_make(acci.hi, acci.lo);
  }

  dd blkr = dd_block_sum(accr);
  dd blki = dd_block_sum(acci);
  dd* part = static_cast<dd*>(a.part);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = blkr;
    part[2 * blockIdx.x + 1] = blki;
  }
  if (!arrive_last(a.counter)) return;
  if (threadIdx.x < 32) {
    dd tr = {0.0, 0.0}, ti = {0.0, 0.0};
    for (unsigned int b = threadIdx.x; b < gridDim.x; b += 32) {
      tr = dd_add(tr, part[2 * b]);
      ti = dd_add(ti, part[2 * b + 1]);
    }
    tr = dd_warp_sum(tr);
    ti = dd_warp_sum(ti);
    if (threadIdx.x == 0) {
      double* out = static_cast<double*>(a.out);
      int32_t st = PERM_OK;
      if (sh.nonfinite) st = PERM_EINVAL;
      else if (sh.bound_log2 + N > 1000) st = PERM_ERANGE;
      else if (*a.aborted) st = stop_status(*a.aborted);
      const double nan = __longlong_as_double(0x7ff8000000000000ll);
      if (a.mode == 0) {
        const double f = (N & 1) ? 2.0 : -2.0;
        out[0] = st != PERM_OK ? nan : (sh.zero_row ? 0.0 : (tr.hi + tr.lo) * f);
        out[1] = st != PERM_OK ? nan : (sh.zero_row ? 0.0 : (ti.hi + ti.lo) * f);
      } else {
        out[0] = st != PERM_OK ? nan : tr.hi;
        out[1] = st != PERM_OK ? 0.0 : tr.lo;
        out[2] = st != PERM_OK ? nan : ti.hi;
        out[3] = st != PERM_OK ? 0.0 : ti.lo;
      }
      if (a.status) *a.status = st;
      *a.counter = 0u;
    }
  }
}

}  // namespace permgpu
