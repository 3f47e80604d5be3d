// Fused permanent gradient: the full n x n matrix G = d perm(A) / dA of one or
// many equally sized matrices in one Gray-code sweep (real and complex, n <= 32).
//
// Derivation (Eq. nwx, x_i = (1/2) sum_l delta_l a_il with delta_l = +1 when
// column l is in the subset or l = n-1, else -1):
//     perm = 2 (-1)^(n-1) sum_g (-1)^g prod_i x_i,
//     G_kl = (-1)^(n-1) sum_g (-1)^g delta_l(g) v_k(g),   v_k = prod_{i != k} x_i.
// With w_k = (-1)^g v_k, T_k = sum_g w_k and U_kl = the sum of w_k over the
// steps where column l is in: G_kl = (-1)^(n-1) (2 U_kl - T_k) for l < n-1 and
// G_{k,n-1} = (-1)^(n-1) T_k.  U is kept with a running prefix P_k of w_k
// inside each aligned chunk: when column j enters at step t, U_kj -= P_k(t-1);
// when it leaves, U_kj += P_k(t-1); at the chunk's end every column still in
// adds P_k.  That is O(n) additions per step (one column flips per step).
//
// GB300 layout:
//  * A sub-group of 8 lanes walks one aligned chunk; lane l owns rows
//    R l .. R l + R - 1 (R = 1..4, the least with 8 R >= n), four sub-groups per warp
//    on four neighbouring chunks.  Rows are staged as in the forward kernels:
//    64-bit fixed point per row with a power-of-two row scale, one exact
//    integer add per row and step.
//  * v_k = prod_{i != k} x_i: products of the R local rows except each one,
//    then an exclusive butterfly over the 8 lanes (xor 1, 2, 4), then one
//    multiply per row: 15 mantissa products per lane and step for R = 4
//    (3.75 per row), on the integer pipes, with 62-bit mantissas and integer
//    exponents (relative error below 2^-58 per term).
//  * Each term is rounded once to binary64 and accumulated into P (FP64 pipe);
//    the column-flip updates of U live in shared memory, only for the columns
//    that flip inside a chunk (j < c); the other columns are constant over the
//    chunk and take P at its end.
//  * At the end of a block-item (16 chunks of one matrix) the CTA folds its 16
//    sub-groups into a per-CTA slot in global memory in a fixed order; a
//    finishing kernel sums the slots in a fixed order (double-double) and
//    forms G.  Results are bitwise reproducible for a given launch shape.
//  * The permanent itself is formed from the gradient by the row expansion
//    perm = sum_l a_0l G_0l (double-double), so it costs nothing in the sweep.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "real.cuh"

namespace permgpu {
namespace {

constexpr int kGL = 8;                  // lanes per sub-group
constexpr int kGWarps = 4;              // warps per CTA
constexpr int kGThreads = 32 * kGWarps;
constexpr int kGSub = kGWarps * 4;      // sub-groups per CTA
constexpr int kDead = -1000000;         // exponent offset of rows that contribute nothing
constexpr int kCsStride = 32;           // ints per matrix in GradArgs::cs (n <= 32)

struct GradArgs {
  const double* A;    // count matrices, n*n scalars each (a scalar is 1 or 2 doubles)
  int n;
  int cq;             // log2 of the chunk a sub-group walks
  uint32_t qc;        // chunks per matrix (2^(n-1-cq))
  uint32_t bipm;      // block-items (16 chunks) per matrix
  uint64_t nbi;       // count * bipm
  uint32_t sb;        // slots per matrix
  double* slots;      // [count][sb][n][8R] scalars, zeroed before the launch
  uint32_t* flags;    // [count]: bit 0 nonfinite, bit 1 range, 8..15 #zero rows, 16..23 first zero row
  const volatile uint32_t* abort_word;  // perm_set_abort_word (device view), or null
  uint64_t budget_ns;                   // perm_set_time_budget, 0: none
  uint32_t* stopped;                    // bit 0: aborted, bit 1: out of time (zeroed)
  int* cs;            // [count][kCsStride]: column scales c_0..c_{n-1}
};

// ------------------------------------------------------------ real values

// |value| = M 2^e with M = m1:m0 in [2^62, 2^63).
struct RE {
  uint32_t m0, m1;
  int e;
};

__device__ __forceinline__ RE mul(RE a, RE b) {
  Prod p;
  p.m0 = a.m0;
  p.m1 = a.m1;
  const uint32_t pos = prod_mul(p, b.m0, b.m1);
  // M_a M_b = v 2^64 and the new mantissa is v 2^(30 - pos)
  return RE{p.m0, p.m1, a.e + b.e + 34 + (int)pos};
}

__device__ __forceinline__ RE shfl_xor(RE x, int d) {
  return RE{__shfl_xor_sync(0xffffffffu, x.m0, d), __shfl_xor_sync(0xffffffffu, x.m1, d),
            __shfl_xor_sync(0xffffffffu, x.e, d)};
}

// |Y| of an odd fixed-point row value, normalised; the sign bit in neg.
__device__ __forceinline__ RE leaf(long long Y, uint32_t& neg) {
  const uint32_t ylo = (uint32_t)(unsigned long long)Y, yhi = (uint32_t)((unsigned long long)Y >> 32);
  const uint32_t m = (uint32_t)((int32_t)yhi >> 31);
  const unsigned long long ay = ((unsigned long long)(yhi ^ m) << 32) | ((ylo ^ m) | 1u);
  const int lz = __clzll((long long)ay);  // >= 2 since |Y| < 2^62
  const unsigned long long nm = ay << (lz - 1);
  neg = m & 1u;
  return RE{(uint32_t)nm, (uint32_t)(nm >> 32), 1 - lz};
}

// sign * M 2^E (E = e + eoff) rounded to binary64 (ties away from zero),
// flushed to zero below the normal range.
__device__ __forceinline__ double to_double(RE v, int eoff, uint32_t signbit) {
  const int f = v.e + eoff + 62 + 1022;  // biased exponent minus one
  uint32_t rlo, rhi;
  asm("add.cc.u32 %0, %2, 512;\n\t"
      "addc.u32 %1, %3, 0;"
      : "=r"(rlo), "=r"(rhi)
      : "r"(v.m0), "r"(v.m1));
  const uint32_t lo32 = __funnelshift_r(rlo, rhi, 10);
  const uint32_t hi32 = (rhi >> 10) + ((uint32_t)min(f, 2045) << 20) + signbit;
  return f < 1 ? 0.0 : __hiloint2double((int)hi32, (int)lo32);
}

// --------------------------------------------------------- complex values

// value = (r + i im) 2^e, r = r1 2^31 + r0 (signed high limb, 31-bit low limb),
// the larger part normalised to [2^60, 2^61].
struct CE {
  int32_t r1, i1;
  uint32_t r0, i0;
  int e;
};

__device__ __forceinline__ CE mul(CE a, CE b) {
  // the limb arithmetic of cprod_mul (complex.cuh), both operands already in
  // limbs: middle partial products (scale 2^31), high ones (scale 2^62),
  // renormalisation of the larger part to 2^60, limb split
  int s;
  asm("{\n\t"
      ".reg .s64 tr, ti, vr, vi;\n\t"
      ".reg .s32 ni1, ni0, vrh, vih, m1, m2, a1, a2, w, pos;\n\t"
      ".reg .u32 ul, uh;\n\t"
      "neg.s32 ni1, %3;\n\t"
      "neg.s32 ni0, %4;\n\t"
      "mul.wide.s32 tr, %1, %6;\n\t"
      "mad.wide.s32 tr, %2, %5, tr;\n\t"
      "mad.wide.s32 tr, ni1, %8, tr;\n\t"
      "mad.wide.s32 tr, ni0, %7, tr;\n\t"
      "mul.wide.s32 ti, %1, %8;\n\t"
      "mad.wide.s32 ti, %2, %7, ti;\n\t"
      "mad.wide.s32 ti, %3, %6, ti;\n\t"
      "mad.wide.s32 ti, %4, %5, ti;\n\t"
      "shr.s64 tr, tr, 31;\n\t"
      "shr.s64 ti, ti, 31;\n\t"
      "mad.wide.s32 vr, %1, %5, tr;\n\t"
      "mad.wide.s32 vr, ni1, %7, vr;\n\t"
      "mad.wide.s32 vi, %1, %7, ti;\n\t"
      "mad.wide.s32 vi, %3, %5, vi;\n\t"
      "mov.b64 {ul, vrh}, vr;\n\t"
      "mov.b64 {ul, vih}, vi;\n\t"
      "shr.s32 m1, vrh, 31;\n\t"
      "xor.b32 a1, vrh, m1;\n\t"
      "shr.s32 m2, vih, 31;\n\t"
      "xor.b32 a2, vih, m2;\n\t"
      "or.b32 w, a1, a2;\n\t"
      "bfind.u32 pos, w;\n\t"
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
      : "=r"(s), "+r"(a.r1), "+r"(a.r0), "+r"(a.i1), "+r"(a.i0)
      : "r"(b.r1), "r"(b.r0), "r"(b.i1), "r"(b.i0));
  return CE{a.r1, a.i1, a.r0, a.i0, a.e + b.e + 62 - s};
}

__device__ __forceinline__ CE shfl_xor(CE x, int d) {
  return CE{__shfl_xor_sync(0xffffffffu, x.r1, d), __shfl_xor_sync(0xffffffffu, x.i1, d),
            __shfl_xor_sync(0xffffffffu, x.r0, d), __shfl_xor_sync(0xffffffffu, x.i0, d),
            __shfl_xor_sync(0xffffffffu, x.e, d)};
}

__device__ __forceinline__ CE leaf(longlong2 Y) {
  const unsigned long long mag = (unsigned long long)((Y.x ^ (Y.x >> 63)) | (Y.y ^ (Y.y >> 63)));
  const int sh = __clzll((long long)mag) - 3;  // top bit to 2^60 (|parts| <= 2^60)
  const long long r = Y.x << sh, im = Y.y << sh;
  return CE{(int32_t)(r >> 31), (int32_t)(im >> 31), (uint32_t)r & 0x7FFFFFFFu, (uint32_t)im & 0x7FFFFFFFu, -sh};
}

// v 2^E for a signed v (|v| <= 2^62) rounded to binary64, flushed below the
// normal range; negated when neg is set.
__device__ __forceinline__ double part_to_double(long long v, int E, uint32_t neg) {
  const unsigned long long s = (unsigned long long)(v >> 63);
  const unsigned long long mag = ((unsigned long long)v ^ s) - s;
  const int lz = __clzll((long long)(mag | 1ull));
  const unsigned long long nm = mag << (lz - 1);  // [2^62, 2^63) unless v == 0
  RE t{(uint32_t)nm, (uint32_t)(nm >> 32), 0};
  const uint32_t sign = ((uint32_t)s ^ (0u - neg)) & 0x80000000u;
  const double d = to_double(t, E - (lz - 1), sign);
  return mag == 0 ? 0.0 : d;
}

// ----------------------------------------------------------- type policy

template <bool CPLX>
struct Val;

template <>
struct Val<false> {
  using Y = long long;
  using E = RE;
  using Acc = double;
  static constexpr int kW = 1;
  __device__ static Acc zero() { return 0.0; }
};

template <>
struct Val<true> {
  using Y = longlong2;
  using E = CE;
  using Acc = double2;
  static constexpr int kW = 2;
  __device__ static Acc zero() { return make_double2(0.0, 0.0); }
};

__device__ __forceinline__ void yadd(long long& y, long long d) { y += d; }
__device__ __forceinline__ void yadd(longlong2& y, longlong2 d) {
  y.x += d.x;
  y.y += d.y;
}
__device__ __forceinline__ double aadd(double a, double b) { return a + b; }
__device__ __forceinline__ double2 aadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
// Sign flips as an integer xor of the high word: one ALU op, so that the
// column-flip update costs a single DADD on the (1/64-rate) FP64 pipe.
__device__ __forceinline__ double aneg(double a, bool neg) {
  const uint32_t m = neg ? 0x80000000u : 0u;
  return __hiloint2double((int)((uint32_t)__double2hiint(a) ^ m), __double2loint(a));
}
__device__ __forceinline__ double2 aneg(double2 a, bool neg) { return make_double2(aneg(a.x, neg), aneg(a.y, neg)); }
__device__ __forceinline__ double asel(double a, bool keep) { return keep ? a : 0.0; }
__device__ __forceinline__ double2 asel(double2 a, bool keep) { return keep ? a : make_double2(0.0, 0.0); }

// ---------------------------------------------------------------- staging

// One matrix into shared memory as signed column increments (both element
// types: Y_i = 2 x_i 2^(s_i), x_i in units of 2^(-s_i - 1)).  Real rows round
// column n-1 to odd multiples (|Y_i| is then never zero, as in the forward
// kernel); padded rows are the constant 1.  Columns far below the largest are
// first scaled by exact powers of two, A' = A diag(2^c) (s_cexp, their sum in
// *s_csum); every minor of A' is 2^(sum c - c_l) times that of A.  The sweep
// takes 2^(-sum c) into its term exponents and the finishing kernel
// multiplies column l by 2^(c_l); the range check is on A itself.
template <bool CPLX>
__device__ void grad_stage(const double* __restrict__ A, int n, int NR, typename Val<CPLX>::Y* D,
                           typename Val<CPLX>::Y* base, int* s_scale, uint32_t* s_flags, int* s_sall,
                           uint32_t* gflags, int* s_cexp, int* s_csum) {
  using Y = typename Val<CPLX>::Y;
  __shared__ int s_bound, s_zc, s_zi;
  const int tid = threadIdx.x;
  const int csum = column_scales<CPLX ? 2 : 1>(A, n, s_cexp, true);
  if (tid == 0) *s_csum = csum;
  if (tid == 0) {
    *s_flags = 0u;
    *s_sall = 0;
    s_bound = 0;
    s_zc = 0;
    s_zi = 255;
  }
  __syncthreads();
  if (tid < n) {
    const int W = CPLX ? 2 : 1;
    const double* row = A + (size_t)tid * n * W;
    double absum = 0.0;
    int fin = 1;
    for (int j = 0; j < n * W; ++j) {
      const double v = row[j];
      fin &= isfinite(v) ? 1 : 0;
      absum += ldexp(fabs(v), s_cexp[j / W]);
    }
    int k = 0;
    if (fin && absum > 0.0) frexp(absum, &k);
    int s;
    if constexpr (CPLX) {
      s = 60 - k;
      long long sr = 0, si = 0;
      for (int j = 0; j < n - 1; ++j) {
        const long long qr = fin ? __double2ll_rn(ldexp(row[2 * j], s + s_cexp[j])) : 0;
        const long long qi = fin ? __double2ll_rn(ldexp(row[2 * j + 1], s + s_cexp[j])) : 0;
        sr += qr;
        si += qi;
        D[(2 * j) * NR + tid] = make_longlong2(2 * qr, 2 * qi);
        D[(2 * j + 1) * NR + tid] = make_longlong2(-2 * qr, -2 * qi);
      }
      const long long nr = fin ? __double2ll_rn(ldexp(row[2 * (n - 1)], s + s_cexp[n - 1])) : 0;
      const long long ni = fin ? __double2ll_rn(ldexp(row[2 * (n - 1) + 1], s + s_cexp[n - 1])) : 0;
      base[tid] = make_longlong2(nr - sr, ni - si);
    } else {
      s = 61 - k;
      long long qsum = 0;
      for (int j = 0; j < n - 1; ++j) {
        const long long q = fin ? __double2ll_rn(ldexp(row[j], s - 1 + s_cexp[j])) : 0;
        qsum += 2 * q;
        D[(2 * j) * NR + tid] = 4 * q;
        D[(2 * j + 1) * NR + tid] = -4 * q;
      }
      const long long qn = fin ? 2 * __double2ll_rd(ldexp(row[n - 1], s - 1 + s_cexp[n - 1])) + 1 : 1;
      base[tid] = qn - qsum;
    }
    s_scale[tid] = s;
    atomicAdd(s_sall, s + 1);
    atomicAdd(&s_bound, k - 1);
    if (!fin) atomicOr(s_flags, 1u);
    if (fin && absum == 0.0) {
      atomicAdd(&s_zc, 1);
      atomicMin(&s_zi, tid);
    }
  } else if (tid < NR) {
    for (int j = 0; j < n - 1; ++j) {
      D[(2 * j) * NR + tid] = Y{};
      D[(2 * j + 1) * NR + tid] = Y{};
    }
    if constexpr (CPLX)
      base[tid] = make_longlong2(1, 0);
    else
      base[tid] = 1;
    s_scale[tid] = -1;
  }
  __syncthreads();
  if (tid == 0) {
    uint32_t f = *s_flags;
    if (s_bound - csum + n > 1000) f |= 2u;
    f |= (uint32_t)min(s_zc, 255) << 8;
    f |= (uint32_t)s_zi << 16;
    *s_flags = f;
    *gflags = f;
  }
  __syncthreads();
}

// ------------------------------------------------------------ main sweep

template <bool CPLX, int R>
__global__ void __launch_bounds__(kGThreads, (CPLX && R == 4) ? 2 : 4) ryser_grad_kernel(GradArgs a) {
  using V = Val<CPLX>;
  using Y = typename V::Y;
  using E = typename V::E;
  using Acc = typename V::Acc;
  constexpr int NR = kGL * R;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_scale[32], s_cexp[64];
  __shared__ uint32_t s_flags;
  __shared__ int s_sall, s_csum;
  const int n = a.n, cq = a.cq;
  Y* D = reinterpret_cast<Y*>(smem);
  Y* base = D + (size_t)2 * (n > 1 ? n - 1 : 0) * NR;
  Acc* U = reinterpret_cast<Acc*>(base + NR);
  Acc* Ps = U + (size_t)kGSub * cq * NR;
  uint64_t* Gs = reinterpret_cast<uint64_t*>(Ps + (size_t)kGSub * NR);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, sg = lane >> 3, l = lane & 7;
  const int sgi = w * 4 + sg;
  const int row0 = l * R;
  const uint32_t gmask = 0xFFu << (8 * sg);
  const int W = V::kW;
  const uint32_t nsteps = 1u << cq;

  uint64_t staged = ~0ull;
  int eoff[R];
  __shared__ uint32_t s_stop[2];  // alternating, so a slot is rewritten only after a barrier
  uint32_t iter = 0;
  const uint64_t t_start = global_ns();
  const bool watch = a.abort_word || a.budget_ns;
  for (uint64_t bi = blockIdx.x; bi < a.nbi; bi += gridDim.x) {
    if (watch) {
      // cancellation and the time budget between block-items, one decision per CTA
      if (tid == 0) {
        uint32_t v = 0u;
        if (a.abort_word && *a.abort_word != 0u) v = 1u;
        else if (a.budget_ns && global_ns() - t_start > a.budget_ns) v = 2u;
        if (v) atomicOr(a.stopped, v);
        s_stop[iter & 1u] = v;
      }
      __syncthreads();
      if (s_stop[iter & 1u]) break;
      ++iter;
    }
    const uint64_t p = bi / a.bipm;
    const uint32_t q = (uint32_t)(bi - p * a.bipm);
    if (p != staged) {
      __syncthreads();
      grad_stage<CPLX>(a.A + p * (uint64_t)n * n * W, n, NR, D, base, s_scale, &s_flags, &s_sall, a.flags + p,
                       s_cexp, &s_csum);
      staged = p;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int i = row0 + r;
        eoff[r] = i < n ? -(s_sall + s_csum - (s_scale[i] + 1)) : kDead;
      }
    }
    // the matrix's column scales, for the finishing kernel (once per matrix)
    if (q == 0 && tid < n) a.cs[p * kCsStride + tid] = s_cexp[tid];
    if (s_flags & 3u) continue;  // the finishing kernels write NaN
    const uint32_t qq = q * 16u + (uint32_t)sgi;
    const bool active = qq < a.qc;
    const uint64_t g0 = active ? (uint64_t)qq << cq : 0;
    int eo[R];
#pragma unroll
    for (int r = 0; r < R; ++r) eo[r] = active ? eoff[r] : kDead;

    Acc* Um = U + (size_t)sgi * cq * NR + row0;
    for (int j = 0; j < cq; ++j) {
#pragma unroll
      for (int r = 0; r < R; ++r) Um[j * NR + r] = V::zero();
    }
    Y y[R];
#pragma unroll
    for (int r = 0; r < R; ++r) y[r] = base[row0 + r];
    const uint64_t G0 = gray64(g0);
    for (int j = (cq > 0 ? cq - 1 : 0); j < n - 1; ++j) {
      if ((G0 >> j) & 1u) {
        const Y* d = D + (size_t)(2 * j) * NR + row0;
#pragma unroll
        for (int r = 0; r < R; ++r) yadd(y[r], d[r]);
      }
    }
    Acc P[R];
#pragma unroll
    for (int r = 0; r < R; ++r) P[r] = V::zero();
    const uint32_t kb = (qq & 1u) << cq;  // bit cq of g: the sign of the chunk's middle step
    const uint32_t gpar0 = (uint32_t)g0 & 1u;

    for (uint32_t t = 0; t < nsteps; ++t) {
      if (t) {
        const int j = __ffs((int)t) - 1;
        const uint32_t sbit = ((t | kb) >> (j + 1)) & 1u;  // 1: column j leaves
        const Y* d = D + (size_t)(2 * j + sbit) * NR + row0;
        Acc* u = Um + j * NR;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          yadd(y[r], d[r]);
          u[r] = aadd(u[r], aneg(P[r], sbit == 0u));
        }
      }
      const uint32_t gs = (t ^ gpar0) & 1u;  // (-1)^g
      E lf[R];
      uint32_t neg = 0u;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if constexpr (CPLX) {
          lf[r] = leaf(y[r]);
        } else {
          uint32_t nb;
          lf[r] = leaf(y[r], nb);
          neg |= nb << r;
        }
      }
      // products of the local rows except each one, and of all of them
      E ex[R], grp;
      if constexpr (R == 1) {
        grp = lf[0];
      } else if constexpr (R == 2) {
        ex[0] = lf[1];
        ex[1] = lf[0];
        grp = mul(lf[0], lf[1]);
      } else if constexpr (R == 3) {
        const E p01 = mul(lf[0], lf[1]);
        ex[0] = mul(lf[1], lf[2]);
        ex[1] = mul(lf[0], lf[2]);
        ex[2] = p01;
        grp = mul(p01, lf[2]);
      } else {
        const E p01 = mul(lf[0], lf[1]), p23 = mul(lf[2], lf[3]);
        ex[0] = mul(lf[1], p23);
        ex[1] = mul(lf[0], p23);
        ex[2] = mul(p01, lf[3]);
        ex[3] = mul(p01, lf[2]);
        grp = mul(p01, p23);
      }
      // exclusive butterfly over the 8 lanes of the sub-group
      E o = shfl_xor(grp, 1);
      grp = mul(grp, o);
      E x2 = shfl_xor(grp, 2);
      o = mul(o, x2);
      grp = mul(grp, x2);
      E x4 = shfl_xor(grp, 4);
      o = mul(o, x4);
      if constexpr (CPLX) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          E v = o;
          if constexpr (R > 1) v = mul(o, ex[r]);
          const int Ev = v.e + eo[r];
          const double vr = part_to_double(((long long)v.r1 << 31) | v.r0, Ev, gs);
          const double vi = part_to_double(((long long)v.i1 << 31) | v.i0, Ev, gs);
          P[r].x += vr;
          P[r].y += vi;
        }
      } else {
        // parity of the negative rows of the sub-group, without this row
        const uint32_t bal = __ballot_sync(0xffffffffu, __popc(neg) & 1);
        const uint32_t gp = (uint32_t)__popc(bal & gmask) & 1u;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          E v = o;
          if constexpr (R > 1) v = mul(o, ex[r]);
          const uint32_t sbit = (gp ^ ((neg >> r) & 1u) ^ gs) << 31;
          P[r] += to_double(v, eo[r], sbit);
        }
      }
    }

    // publish the chunk's P and Gray codes, then fold the 16 sub-groups
#pragma unroll
    for (int r = 0; r < R; ++r) Ps[(size_t)sgi * NR + row0 + r] = P[r];
    if (l == 0) {
      Gs[2 * sgi] = gray64(g0);
      Gs[2 * sgi + 1] = gray64(g0 + nsteps - 1);
    }
    __syncthreads();
    Acc* slot = reinterpret_cast<Acc*>(a.slots) + ((size_t)p * a.sb + q % a.sb) * (size_t)n * NR;
    for (int e = tid; e < n * NR; e += kGThreads) {
      const int j = e / NR, i = e - j * NR;
      if (i >= n) continue;
      Acc s = V::zero();
      for (int k = 0; k < kGSub; ++k) {
        const Acc pk = Ps[(size_t)k * NR + i];
        if (j == n - 1) {
          s = aadd(s, pk);
        } else if (j < cq) {
          s = aadd(s, aadd(U[((size_t)k * cq + j) * NR + i], asel(pk, (Gs[2 * k + 1] >> j) & 1u)));
        } else {
          s = aadd(s, asel(pk, (Gs[2 * k] >> j) & 1u));
        }
      }
      slot[e] = aadd(slot[e], s);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------- finishing

struct FinishArgs {
  const double* A;
  int n, NR, count;
  uint32_t sb;
  const double* slots;
  const uint32_t* flags;
  double* G;
  double* out;
  uint32_t* status_bits;  // [0]: EINVAL / ERANGE bits, [1]: the sweep's stop bits
  const int* cs;          // GradArgs::cs
};

// G for column j of matrix p (grid: count x n, 256 threads): warp w sums slots
// w, w + 8, ... in a fixed order (double-double), lane = row.
template <bool CPLX>
__global__ void __launch_bounds__(256) grad_finish_kernel(FinishArgs f) {
  constexpr int W = CPLX ? 2 : 1;
  const int j = blockIdx.y, n = f.n, NR = f.NR;
  const uint64_t p = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  __shared__ dd s_u[8][W][32], s_t[8][W][32];
  dd u[W], t[W];
  for (int c = 0; c < W; ++c) u[c] = t[c] = dd{0.0, 0.0};
  if (lane < n) {
    const double* base = f.slots + (size_t)p * f.sb * n * NR * W;
    for (uint32_t s = w; s < f.sb; s += 8) {
      const double* sl = base + (size_t)s * n * NR * W;
      for (int c = 0; c < W; ++c) {
        u[c] = dd_add_d(u[c], sl[((size_t)j * NR + lane) * W + c]);
        t[c] = dd_add_d(t[c], sl[((size_t)(n - 1) * NR + lane) * W + c]);
      }
    }
  }
  for (int c = 0; c < W; ++c) {
    s_u[w][c][lane] = u[c];
    s_t[w][c][lane] = t[c];
  }
  __syncthreads();
  if (w != 0 || lane >= n) return;
  const uint32_t fl = f.flags[p];
  const int zc = (fl >> 8) & 0xFF, zi = (fl >> 16) & 0xFF;
  const double sg = ((n - 1) & 1) ? -1.0 : 1.0;
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  for (int c = 0; c < W; ++c) {
    dd U = {0.0, 0.0}, T = {0.0, 0.0};
    for (int k = 0; k < 8; ++k) {
      U = dd_add(U, s_u[k][c][lane]);
      T = dd_add(T, s_t[k][c][lane]);
    }
    double g;
    if (j == n - 1) {
      g = sg * (T.hi + T.lo);
    } else {
      const dd d = dd_add(dd{2.0 * U.hi, 2.0 * U.lo}, dd{-T.hi, -T.lo});
      g = sg * (d.hi + d.lo);
    }
    // undo the column scales: the sweep summed 2^(-sum c) G'_kj, and
    // G_kj = 2^(c_j - sum c) G'_kj (exact unless it underflows)
    g = ldexp(g, f.cs[p * kCsStride + j]);
    if ((fl & 3u) || f.status_bits[1]) g = nan;
    else if (zc >= 2 || (zc == 1 && lane != zi)) g = 0.0;
    f.G[((size_t)p * n * n + (size_t)lane * n + j) * W + c] = g;
  }
}

// perm = sum_l a_0l G_0l (row expansion) in double-double, one warp per matrix.
__device__ __forceinline__ dd two_prod(double a, double b) {
  const double p = a * b;
  return dd{p, fma(a, b, -p)};
}

template <bool CPLX>
__global__ void __launch_bounds__(256) grad_perm_kernel(FinishArgs f) {
  const int lane = threadIdx.x & 31;
  const uint64_t p = (uint64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (p >= (uint64_t)f.count) return;
  const int n = f.n;
  constexpr int W = CPLX ? 2 : 1;
  const double* A = f.A + p * (uint64_t)n * n * W;
  const double* G = f.G + p * (uint64_t)n * n * W;
  dd re = {0.0, 0.0}, im = {0.0, 0.0};
  if (lane < n) {
    if constexpr (CPLX) {
      const double ar = A[2 * lane], ai = A[2 * lane + 1], gr = G[2 * lane], gi = G[2 * lane + 1];
      re = dd_add(two_prod(ar, gr), two_prod(-ai, gi));
      im = dd_add(two_prod(ar, gi), two_prod(ai, gr));
    } else {
      re = two_prod(A[lane], G[lane]);
    }
  }
  re = dd_warp_sum(re);
  if (CPLX) im = dd_warp_sum(im);
  if (lane != 0) return;
  const uint32_t fl = f.flags[p];
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  double vr = re.hi + re.lo, vi = im.hi + im.lo;
  if ((fl & 3u) || f.status_bits[1]) vr = vi = nan;
  else if ((fl >> 8) & 0xFF) vr = vi = 0.0;
  f.out[p * W] = vr;
  if (CPLX) f.out[p * W + 1] = vi;
  if (fl & 3u) atomicOr(f.status_bits, fl & 3u);
}

__global__ void grad_status_kernel(const uint32_t* bits, int32_t* status) {
  const uint32_t b = bits[0];
  if (status) *status = (b & 1u) ? PERM_EINVAL : (b & 2u) ? PERM_ERANGE : stop_status(bits[1]);
}

// n = 0: the empty product (perm = 1, no gradient entries).
__global__ void grad_empty_kernel(double* out, int count, int W, int32_t* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) {
    out[(size_t)i * W] = 1.0;
    if (W == 2) out[(size_t)i * W + 1] = 0.0;
  }
  if (i == 0 && status) *status = PERM_OK;
}

// Mixed sizes: gather the matrices of one order into a contiguous batch and
// scatter its results back (one CTA per matrix).
__global__ void grad_gather_kernel(const double* __restrict__ src, const int64_t* __restrict__ offs, int nn_w,
                                   double* __restrict__ dst) {
  const int m = blockIdx.x;
  const double* s = src + offs[m];
  double* d = dst + (size_t)m * nn_w;
  for (int i = threadIdx.x; i < nn_w; i += blockDim.x) d[i] = s[i];
}

__global__ void grad_scatter_kernel(const double* __restrict__ G, const double* __restrict__ out, const int64_t* offs,
                                    const int64_t* out_idx, int nn_w, int W, double* __restrict__ Gdst,
                                    double* __restrict__ outdst) {
  const int m = blockIdx.x;
  const double* s = G + (size_t)m * nn_w;
  double* d = Gdst + offs[m];
  for (int i = threadIdx.x; i < nn_w; i += blockDim.x) d[i] = s[i];
  if (threadIdx.x < W) outdst[out_idx[m] * W + threadIdx.x] = out[(size_t)m * W + threadIdx.x];
}

// status of a mixed call: the first failing group's code, else PERM_OK
__global__ void grad_status_merge_kernel(const int32_t* st, int groups, int32_t* status) {
  int32_t r = PERM_OK;
  for (int g = 0; g < groups; ++g)
    if (r == PERM_OK && st[g] != PERM_OK) r = st[g];
  if (status) *status = r;
}

// ------------------------------------------------------------------ host

using KernelFn = void (*)(GradArgs);

KernelFn grad_kernel(bool cplx, int R) {
  if (cplx)
    return R == 1   ? ryser_grad_kernel<true, 1>
           : R == 2 ? ryser_grad_kernel<true, 2>
           : R == 3 ? ryser_grad_kernel<true, 3>
                    : ryser_grad_kernel<true, 4>;
  return R == 1   ? ryser_grad_kernel<false, 1>
         : R == 2 ? ryser_grad_kernel<false, 2>
         : R == 3 ? ryser_grad_kernel<false, 3>
                  : ryser_grad_kernel<false, 4>;
}

size_t grad_smem(bool cplx, int n, int R, int cq) {
  const size_t NR = (size_t)kGL * R;
  const size_t ys = cplx ? 16 : 8, as = cplx ? 16 : 8;
  return ys * (2 * (size_t)(n > 1 ? n - 1 : 0) * NR + NR) + as * ((size_t)kGSub * cq * NR + (size_t)kGSub * NR) +
         sizeof(uint64_t) * 2 * kGSub;
}

int ceil_log2_u64(uint64_t v) {
  int k = 0;
  while ((1ull << k) < v) ++k;
  return k;
}

// SM count of the device and, once per device and kernel, the opt-in shared
// memory limit set on all six sweep kernels.
int device_prepare(int dev) {
  static std::mutex mu;
  static int sms_cache[64] = {0};
  std::lock_guard<std::mutex> lock(mu);
  if (dev < 0 || dev >= 64) return 0;
  if (!sms_cache[dev]) {
    int v = 0, optin = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    // the dynamic limit plus the kernel's static shared memory must stay
    // within the opt-in maximum
    for (int c = 0; c < 2; ++c)
      for (int R = 1; R <= 4; ++R) {
        const void* fn = reinterpret_cast<const void*>(grad_kernel(c != 0, R));
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess ||
            cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)fa.sharedSizeBytes) != cudaSuccess) {
          cudaGetLastError();
          return 0;
        }
      }
    sms_cache[dev] = v;
  }
  return sms_cache[dev];
}

}  // namespace
}  // namespace permgpu

using namespace permgpu;

namespace permgpu {
namespace {

// Launch shape and workspace of one equal-order gradient sweep.
struct GradCfg {
  int n = 0, count = 0, R = 1, cq = 0, grid = 0;
  bool cplx = false;
  uint32_t qc = 0, bipm = 0, sb = 0;
  uint64_t nbi = 0;
  size_t smem = 0, slot_doubles = 0, ws_bytes = 0;
  KernelFn fn = nullptr;
};

// n >= 1, count >= 1.
int grad_configure(int n, int count, bool cplx, GradCfg& g) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PERM_ECUDA;
  const int sms = device_prepare(dev);
  if (sms <= 0) return PERM_ECUDA;
  const int W = cplx ? 2 : 1;
  g.n = n;
  g.count = count;
  g.cplx = cplx;
  g.R = n <= 8 ? 1 : n <= 16 ? 2 : n <= 24 ? 3 : 4;
  const int NR = kGL * g.R;
  g.fn = grad_kernel(cplx, g.R);
  // chunk length: the largest cq <= 9 that keeps 4 CTAs (cplx R=4: 2) per SM
  // resident, then shortened so that small batches still fill the GPU
  int cq_max = 0, ctas = 0;
  {
    const int want = (cplx && g.R == 4) ? 2 : 4;
    for (int c = 9; c >= 0; --c) {
      const size_t sm = grad_smem(cplx, n, g.R, c);
      int nb = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, g.fn, kGThreads, sm) != cudaSuccess) {
        cudaGetLastError();
        return PERM_ECUDA;
      }
      if (nb >= want || c == 0) {
        cq_max = c;
        ctas = nb;
        break;
      }
    }
  }
  if (ctas <= 0) return PERM_ECUDA;
  const uint64_t B_full = (uint64_t)sms * ctas;
  const uint64_t per_matrix = (2 * B_full + (uint64_t)count - 1) / (uint64_t)count;  // block-items wanted
  int cq = (n - 1) - 4 - ceil_log2_u64(per_matrix);
  cq = cq < 4 ? 4 : cq;
  cq = cq > cq_max ? cq_max : cq;
  if (cq > n - 5) cq = n - 5 > 0 ? n - 5 : 0;
  g.cq = cq;
  g.qc = 1u << (n - 1 - cq);
  g.bipm = g.qc >= 16 ? g.qc / 16 : 1;
  g.nbi = (uint64_t)count * g.bipm;
  g.grid = (int)(g.nbi < B_full ? g.nbi : B_full);
  g.sb = g.bipm < (uint32_t)g.grid ? g.bipm : (uint32_t)g.grid;
  g.slot_doubles = (size_t)count * g.sb * n * NR * W;
  g.ws_bytes = sizeof(double) * g.slot_doubles + sizeof(uint32_t) * ((size_t)count + 4) +
               sizeof(int) * (size_t)count * kCsStride;
  g.smem = grad_smem(cplx, n, g.R, cq);
  return PERM_OK;
}

// The sweep and its finishing kernels on a caller-provided workspace of
// g.ws_bytes (cleared here, on the stream).  Allocates nothing.
int grad_launch(const GradCfg& g, const void* A, void* out, void* G, int32_t* status, void* ws, cudaStream_t s) {
  double* slots = static_cast<double*>(ws);
  uint32_t* flags = reinterpret_cast<uint32_t*>(slots + g.slot_doubles);
  uint32_t* bits = flags + g.count;
  int* cs = reinterpret_cast<int*>(bits + 4);
  if (cudaMemsetAsync(ws, 0, g.ws_bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return PERM_ECUDA;
  }
  GradArgs ga;
  memset(&ga, 0, sizeof(ga));
  ga.A = static_cast<const double*>(A);
  ga.n = g.n;
  ga.cq = g.cq;
  ga.qc = g.qc;
  ga.bipm = g.bipm;
  ga.nbi = g.nbi;
  ga.sb = g.sb;
  ga.slots = slots;
  ga.flags = flags;
  ga.abort_word = current_abort_word();
  ga.budget_ns = current_time_budget();
  ga.stopped = bits + 1;
  ga.cs = cs;
  void* params[] = {&ga};
  cudaError_t e =
      cudaLaunchKernel(reinterpret_cast<const void*>(g.fn), dim3(g.grid), dim3(kGThreads), params, g.smem, s);
  FinishArgs fa;
  memset(&fa, 0, sizeof(fa));
  fa.A = static_cast<const double*>(A);
  fa.n = g.n;
  fa.NR = kGL * g.R;
  fa.count = g.count;
  fa.sb = g.sb;
  fa.slots = slots;
  fa.flags = flags;
  fa.G = static_cast<double*>(G);
  fa.out = static_cast<double*>(out);
  fa.status_bits = bits;
  fa.cs = cs;
  if (e == cudaSuccess) {
    if (g.cplx)
      grad_finish_kernel<true><<<dim3(g.count, g.n), 256, 0, s>>>(fa);
    else
      grad_finish_kernel<false><<<dim3(g.count, g.n), 256, 0, s>>>(fa);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    const unsigned pb = (unsigned)((g.count + 7) / 8);
    if (g.cplx)
      grad_perm_kernel<true><<<pb, 256, 0, s>>>(fa);
    else
      grad_perm_kernel<false><<<pb, 256, 0, s>>>(fa);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    grad_status_kernel<<<1, 1, 0, s>>>(bits, status);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return PERM_ECUDA;
  }
  return PERM_OK;
}

}  // namespace
}  // namespace permgpu

extern "C" int perm_grad_batched(const void* A, int n, int count, int type, void* out, void* G, int32_t* status,
                                 void* stream) {
  if (type != PERM_F64 && type != PERM_C128) return PERM_EINVAL;
  if (n < 0 || n > 32) return PERM_ERANGE;
  if (count < 0) return PERM_EINVAL;
  if (count == 0) return status ? (cudaMemsetAsync(status, 0, sizeof(int32_t), (cudaStream_t)stream) == cudaSuccess
                                       ? PERM_OK
                                       : PERM_ECUDA)
                                : PERM_OK;
  if (!out || (n > 0 && (!A || !G))) return PERM_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool cplx = type == PERM_C128;
  const int W = cplx ? 2 : 1;
  if (n == 0) {
    grad_empty_kernel<<<(count + 255) / 256, 256, 0, s>>>(static_cast<double*>(out), count, W, status);
    return cudaGetLastError() == cudaSuccess ? PERM_OK : PERM_ECUDA;
  }
  GradCfg g;
  int rc = grad_configure(n, count, cplx, g);
  if (rc) return rc;
  void* ws = nullptr;
  if (cudaMallocAsync(&ws, g.ws_bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return PERM_ENOMEM;
  }
  rc = grad_launch(g, A, out, G, status, ws, s);
  if (cudaFreeAsync(ws, s) != cudaSuccess && rc == PERM_OK) rc = PERM_ECUDA;
  if (rc) cudaGetLastError();
  return rc;
}

extern "C" int perm_grad(const void* A, int n, int type, void* out, void* G, int32_t* status, void* stream) {
  return perm_grad_batched(A, n, 1, type, out, G, status, stream);
}

// A mixed-order gradient plan: the matrices grouped by order, each group
// gathered into a contiguous batch, swept by one equal-order launch and
// scattered back.  Every device buffer is allocated once, at creation.
struct perm_grad_plan {
  struct Group {
    int n = 0, cnt = 0;
    GradCfg cfg;
    double* Ag = nullptr;  // gathered matrices, then G, then out
    double* Gg = nullptr;
    double* og = nullptr;
    int64_t* offs = nullptr;  // element offsets in A_packed / G_packed (scalars x W)
    int64_t* oidx = nullptr;  // output index of every matrix
  };
  int type = PERM_F64;
  int count = 0;
  std::vector<Group> groups;
  void* buf = nullptr;   // one allocation: group buffers, index arrays, statuses
  void* ws = nullptr;    // sweep workspace, shared by the groups (stream-ordered)
  int32_t* gst = nullptr;
};

static void grad_plan_free(perm_grad_plan* p) {
  if (!p) return;
  cudaFree(p->buf);
  cudaFree(p->ws);
  delete p;
}

extern "C" int perm_grad_plan_create(perm_grad_plan** plan, int type, const int* ns_host, int count,
                                     const int64_t* offsets_host) {
  if (!plan) return PERM_EINVAL;
  *plan = nullptr;
  if (type != PERM_F64 && type != PERM_C128) return PERM_EINVAL;
  if (count < 0 || (count > 0 && (!ns_host || !offsets_host))) return PERM_EINVAL;
  const int W = type == PERM_C128 ? 2 : 1;
  std::vector<std::vector<int>> members(33);
  for (int m = 0; m < count; ++m) {
    const int n = ns_host[m];
    if (n < 0 || n > 32) return PERM_ERANGE;
    if (offsets_host[m] < 0) return PERM_EINVAL;
    members[n].push_back(m);
  }
  perm_grad_plan* p = new perm_grad_plan();
  p->type = type;
  p->count = count;
  size_t doubles = 0, words = 0, ws_max = 0;
  for (int n = 0; n <= 32; ++n) {
    if (members[n].empty()) continue;
    perm_grad_plan::Group g;
    g.n = n;
    g.cnt = (int)members[n].size();
    if (n > 0) {
      int rc = grad_configure(n, g.cnt, type == PERM_C128, g.cfg);
      if (rc) {
        grad_plan_free(p);
        return rc;
      }
      ws_max = std::max(ws_max, g.cfg.ws_bytes);
    }
    doubles += (size_t)g.cnt * ((size_t)n * n * W * 2 + W);
    words += 2 * (size_t)g.cnt;
    p->groups.push_back(g);
  }
  const size_t bytes = sizeof(double) * doubles + sizeof(int64_t) * words + sizeof(int32_t) * (p->groups.size() + 1);
  if (cudaMalloc(&p->buf, bytes) != cudaSuccess || (ws_max && cudaMalloc(&p->ws, ws_max) != cudaSuccess)) {
    cudaGetLastError();
    grad_plan_free(p);
    return PERM_ENOMEM;
  }
  double* d = static_cast<double*>(p->buf);
  int64_t* idx = reinterpret_cast<int64_t*>(d + doubles);
  p->gst = reinterpret_cast<int32_t*>(idx + words);
  std::vector<int64_t> hidx(words);
  size_t ioff = 0;
  for (perm_grad_plan::Group& g : p->groups) {
    const size_t nn_w = (size_t)g.n * g.n * W;
    g.Ag = d;
    g.Gg = d + (size_t)g.cnt * nn_w;
    g.og = g.Gg + (size_t)g.cnt * nn_w;
    d = g.og + (size_t)g.cnt * W;
    g.offs = idx + ioff;
    g.oidx = g.offs + g.cnt;
    const std::vector<int>& ms = members[g.n];
    for (int k = 0; k < g.cnt; ++k) {
      hidx[ioff + k] = offsets_host[ms[k]] * W;
      hidx[ioff + g.cnt + k] = ms[k];
    }
    ioff += 2 * (size_t)g.cnt;
  }
  if (words && cudaMemcpy(idx, hidx.data(), sizeof(int64_t) * words, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    grad_plan_free(p);
    return PERM_ECUDA;
  }
  *plan = p;
  return PERM_OK;
}

extern "C" int perm_grad_plan_run(perm_grad_plan* p, const void* A_packed, void* out, void* G_packed,
                                  int32_t* status, void* stream) {
  if (!p) return PERM_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (p->count == 0)
    return status ? (cudaMemsetAsync(status, 0, sizeof(int32_t), s) == cudaSuccess ? PERM_OK : PERM_ECUDA)
                  : PERM_OK;
  if (!out) return PERM_EINVAL;
  const int W = p->type == PERM_C128 ? 2 : 1;
  int rc = PERM_OK;
  for (size_t gi = 0; gi < p->groups.size() && rc == PERM_OK; ++gi) {
    const perm_grad_plan::Group& g = p->groups[gi];
    const int nn_w = g.n * g.n * W;
    if (g.n > 0 && (!A_packed || !G_packed)) return PERM_EINVAL;
    if (g.n > 0) {
      grad_gather_kernel<<<g.cnt, 128, 0, s>>>(static_cast<const double*>(A_packed), g.offs, nn_w, g.Ag);
      if (cudaGetLastError() != cudaSuccess) rc = PERM_ECUDA;
      if (rc == PERM_OK) rc = grad_launch(g.cfg, g.Ag, g.og, g.Gg, p->gst + gi, p->ws, s);
    } else {
      grad_empty_kernel<<<(g.cnt + 255) / 256, 256, 0, s>>>(g.og, g.cnt, W, p->gst + gi);
      if (cudaGetLastError() != cudaSuccess) rc = PERM_ECUDA;
    }
    if (rc == PERM_OK) {
      grad_scatter_kernel<<<g.cnt, 128, 0, s>>>(g.Gg, g.og, g.offs, g.oidx, nn_w, W, static_cast<double*>(G_packed),
                                                static_cast<double*>(out));
      if (cudaGetLastError() != cudaSuccess) rc = PERM_ECUDA;
    }
  }
  if (rc == PERM_OK) {
    grad_status_merge_kernel<<<1, 1, 0, s>>>(p->gst, (int)p->groups.size(), status);
    if (cudaGetLastError() != cudaSuccess) rc = PERM_ECUDA;
  }
  if (rc != PERM_OK) cudaGetLastError();
  return rc;
}

extern "C" void perm_grad_plan_destroy(perm_grad_plan* plan) { grad_plan_free(plan); }

extern "C" int perm_grad_batched_mixed(int type, const int* ns_host, int count, const void* A_packed,
                                       const int64_t* offsets_host, void* out, void* G_packed, int32_t* status,
                                       void* stream) {
  if (type != PERM_F64 && type != PERM_C128) return PERM_EINVAL;
  if (count < 0 || (count > 0 && (!ns_host || !offsets_host || !out))) return PERM_EINVAL;
  for (int m = 0; m < count; ++m)
    if (ns_host[m] > 0 && (!A_packed || !G_packed)) return PERM_EINVAL;
  perm_grad_plan* p = nullptr;
  int rc = perm_grad_plan_create(&p, type, ns_host, count, offsets_host);
  if (rc) return rc;
  rc = perm_grad_plan_run(p, A_packed, out, G_packed, status, stream);
  // the plan's buffers are released after the stream's work on them
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess && rc == PERM_OK) rc = PERM_ECUDA;
  grad_plan_free(p);
  if (rc != PERM_OK) cudaGetLastError();
  return rc;
}
