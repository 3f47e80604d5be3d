// Batched permanents (complex or real): thousands of k x k matrices of uneven
// sizes in one CUDA-graph replay (prep kernel, one persistent work-queue kernel,
// finish kernel).  Each matrix is the Ryser / Nijenhuis-Wilf sweep of the
// single-matrix complex kernel (Alg. 1 over complex entries, chunked as
// Alg. 3 with power-of-two chunks, Sec. 3.1.1):
//
//  * The plan (host) groups matrices by size k and builds a work queue:
//    small k run one matrix per lane (32 matrices of equal k per warp item,
//    the lanes walk the same Gray sequence), large k are cut into aligned
//    chunks of 2^c steps, 32 chunks per warp item.  Items are ordered longest
//    first (LPT) and warps pop them from one atomic counter.
//  * The chunk exponent and the lane/warp mode of every size class come from
//    a heuristic or from perm_batched_autotune, which times the candidates
//    on the plan's own matrices.
//  * Real matrices run the integer product chains of the single-matrix real
//    kernel (odd fixed-point rows, 62-bit mantissas), complex ones those of
//    the complex kernel.
//  * The prep kernel rounds every matrix once to fixed point (as the
//    single-matrix kernel) into a plan-owned table that the main kernel reads
//    through L1 (column reads are warp broadcasts in the chunked mode).
//  * Every item writes its partial to its own slot; the finish kernel adds a
//    matrix's slots in a fixed order (deterministic), scales by 2 (-1)^(k-1)
//    and writes the result.  Execution allocates nothing.
//  * Repeated rows (boson-sampling submatrices drawn with replacement): when
//    the caller labels equal rows, a matrix whose distinct rows rho occur
//    mu_rho times is swept in its transposed form.  Glynn's form of Eq. 2,
//    perm = 2^(1-k) sum_{d, d_f = 1} prod_r d_r prod_j sum_r d_r a_rj, is
//    grouped by the number k_rho of copies of each row with d = -1: the
//    copies contribute (mu_rho - 2 k_rho) row_rho to every column sum, with
//    weight C(mu_rho, k_rho) (-1)^(k_rho).  One copy of a singleton row is
//    fixed at d = +1, the other singletons are the Gray-code bits, and each
//    combination (k_rho) of the repeated rows is one ordinary sweep with a
//    shifted base vector and a weight applied when the slots are added:
//    1/2 prod_rho (mu_rho + 1) terms instead of 2^(k-1).
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "complex.cuh"
#include "kernels.h"
#include "real.cuh"

namespace permgpu {

constexpr int kBatchKMax = 32;
constexpr int kLaneMode = 1, kWarpMode = 0;

// One sweep unit: a matrix, or one multiplicity combination of a matrix with
// repeated rows.
struct BatchMat {
  int32_t k;
  int32_t sum_s;
  int32_t flags;  // 1: non-finite entry or unequal labelled rows, 2: zero row, 4: exponent range
  int32_t slot0;  // first partial slot of this unit
  int64_t a_off;  // element offset of the matrix in the packed input
  int64_t d_off;  // longlong2 offset of its column increments D (shared by a matrix's units)
  int64_t b_off;  // longlong2 offset of its base and zero vectors
  int32_t g;      // Gray bits of the sweep: k - 1 for a plain matrix
  int32_t desc;   // -1: plain (rows of A are the factors); else the unit's descriptor
  int32_t chk;    // -1, or the offset of P, (a, b) x P: labelled rows a, b that must be equal
};

// Descriptor of a transposed unit (ints, host-built): the fixed row f, the G
// toggled rows and R (row, coefficient) pairs of the repeated rows:
// f, G, t_0..t_{G-1}, R, (r, c) x R.  The factors are the columns of A.  The
// units of one matrix share D; the first of them (the one with the equality
// checks, chk >= 0) writes it.

// One output matrix: its units and its slots (contiguous).
struct BatchOut {
  int32_t k;
  int32_t u0, nu;
  int32_t slot0, nslots;
  int32_t pad;
};

struct BatchItem {
  int32_t mode;   // kLaneMode or kWarpMode
  int32_t k;
  int32_t c;      // chunk exponent (warp mode)
  int32_t count;  // lane mode: matrices in this item (<= 32)
  int32_t mat;    // lane mode: first index into lane_mats; warp mode: the matrix
  int32_t slot;   // warp mode: the partial slot of this item
  int64_t chunk0; // warp mode: first chunk
};

struct BatchArgs {
  const double* A;        // packed (re, im) pairs
  const BatchMat* mats;   // units
  const BatchOut* outs;   // output matrices
  const int32_t* desc;    // descriptors of transposed units
  const double* slot_w;   // weight of every slot's partial
  const BatchItem* items;
  const int32_t* lane_mats;
  longlong2* table;
  dd* slots;              // 2 per slot (re, im)
  unsigned int* counter;
  double* out;            // (re, im) per matrix
  int32_t* status;        // per matrix (optional)
  const volatile uint32_t* abort_word;  // perm_set_abort_word (device view), or null
  unsigned int* stopped;  // bit 0: aborted, bit 1: out of time (zeroed before the launch)
  uint64_t budget_ns;     // perm_set_time_budget, 0: none
  int nmats;              // output matrices
  int nunits;
  int nitems;
  int type;               // PERM_C128 or PERM_F64
};

// Column i of the labelled row pairs at chk: 1 if some pair differs there.
__device__ __forceinline__ int batch_labels_differ(const BatchArgs& a, const BatchMat& bm, int i) {
  if (bm.chk < 0) return 0;
  const int32_t* pp = a.desc + bm.chk;
  const int P = pp[0];
  const int w = a.type == PERM_F64 ? 1 : 2;
  const double* col = a.A + (int64_t)w * (bm.a_off + i);
  int bad = 0;
  for (int t = 0; t < P; ++t)
    for (int q = 0; q < w; ++q)
      bad |= col[(int64_t)w * pp[1 + 2 * t] * bm.k + q] != col[(int64_t)w * pp[2 + 2 * t] * bm.k + q];
  return bad;
}

// Transposed unit: factor i is column i of A; the toggles are rows, the
// base holds the fixed row and the repeated rows times their coefficients.
// Scales, rounding and the odd fixed row (real) follow the plain branch; row r
// of A is scaled by 2^cexp[r] (equal rows get equal scales).
__device__ void batch_prep_transposed(const BatchArgs& a, const BatchMat& bm, int& s_sum, int& s_bound,
                                      int& s_flags, const int* cexp) {
  const int k = bm.k;
  const int32_t* d = a.desc + bm.desc;
  const int f = d[0], G = d[1];
  const int32_t* tg = d + 2;
  const int R = d[2 + G];
  const int32_t* rp = d + 3 + G;
  const int i = threadIdx.x;
  if (i >= k) return;
  const bool real = a.type == PERM_F64;
  const int w = real ? 1 : 2;
  const double* col = a.A + (int64_t)w * (bm.a_off + i);  // entry (r, i) at col[w r k]
  double absum = 0.0;
  int fin = 1;
  for (int r = 0; r < k; ++r)
    for (int q = 0; q < w; ++q) {
      const double v = col[(int64_t)w * r * k + q];
      fin &= isfinite(v) ? 1 : 0;
      absum += ldexp(fabs(v), cexp[r]);
    }
  const int bad = batch_labels_differ(a, bm, i);
  int kk = 0;
  if (fin && absum > 0.0) frexp(absum, &kk);
  const bool wd = bm.chk >= 0;
  if (real) {
    long long* RD = reinterpret_cast<long long*>(a.table + bm.d_off);
    long long* rbase = reinterpret_cast<long long*>(a.table + bm.b_off);
    const int s = 61 - kk;
    auto q_of = [&](int r) { return fin ? __double2ll_rn(ldexp(col[(int64_t)r * k], s - 1 + cexp[r])) : 0ll; };
    long long b = fin ? 2 * __double2ll_rd(ldexp(col[(int64_t)f * k], s - 1 + cexp[f])) + 1 : 1;
    for (int j = 0; j < k - 1; ++j) {
      const long long q = j < G ? q_of(tg[j]) : 0;
      b -= 2 * q;
      if (wd) {
        RD[(2 * j) * k + i] = 4 * q;
        RD[(2 * j + 1) * k + i] = -4 * q;
      }
    }
    for (int t = 0; t < R; ++t) b += (long long)rp[2 * t + 1] * 2 * q_of(rp[2 * t]);
    rbase[i] = b;
    rbase[k + i] = 0;
    atomicAdd(&s_sum, s);
  } else {
    longlong2* D = a.table + bm.d_off;
    longlong2* base = a.table + bm.b_off;
    const int s = 60 - kk;
    auto q_of = [&](int r, int part) {
      return fin ? __double2ll_rn(ldexp(col[(int64_t)2 * r * k + part], s + cexp[r])) : 0ll;
    };
    long long br = q_of(f, 0), bi = q_of(f, 1);
    for (int j = 0; j < k - 1; ++j) {
      const long long qr = j < G ? q_of(tg[j], 0) : 0, qi = j < G ? q_of(tg[j], 1) : 0;
      br -= qr;
      bi -= qi;
      if (wd) {
        D[(2 * j) * k + i] = make_longlong2(2 * qr, 2 * qi);
        D[(2 * j + 1) * k + i] = make_longlong2(-2 * qr, -2 * qi);
      }
    }
    for (int t = 0; t < R; ++t) {
      br += (long long)rp[2 * t + 1] * q_of(rp[2 * t], 0);
      bi += (long long)rp[2 * t + 1] * q_of(rp[2 * t], 1);
    }
    base[i] = make_longlong2(br, bi);
    base[k + i] = make_longlong2(0, 0);
    atomicAdd(&s_sum, s);
  }
  atomicAdd(&s_bound, kk - 1);
  if (!fin || bad) atomicOr(&s_flags, 1);
  if (fin && absum == 0.0) atomicOr(&s_flags, 2);
}

// One CTA per unit: D[(2j+s) k + i], base[k], zero[k] as in cplx_stage.
__global__ void __launch_bounds__(kBlock) batch_prep_kernel(BatchArgs a) {
  const int m = blockIdx.x;
  if (m >= a.nunits) return;
  const BatchMat bm = a.mats[m];
  const int k = bm.k;
  longlong2* D = a.table + bm.d_off;
  longlong2* base = a.table + bm.b_off;
  longlong2* zero = base + k;
  __shared__ int s_sum, s_bound, s_flags, s_cexp[64];
  if (threadIdx.x == 0) {
    s_sum = 0;
    s_bound = 0;
    s_flags = 0;
  }
  __syncthreads();
  const int i = threadIdx.x;
  // exact equilibration of the toggled lines (columns; rows of a transposed
  // unit): the sweep sums 2^(sum c) perm, undone through sum_s
  const bool tr = bm.desc >= 0;
  const int csum = a.type == PERM_F64 ? column_scales<1>(a.A + bm.a_off, k, s_cexp, true, tr)
                                      : column_scales<2>(a.A + 2 * bm.a_off, k, s_cexp, true, tr);
  if (tr) {
    batch_prep_transposed(a, bm, s_sum, s_bound, s_flags, s_cexp);
  } else if (a.type == PERM_F64) {
    // real: odd fixed-point rows as in real_stage (Y = 2 x 2^s)
    long long* RD = reinterpret_cast<long long*>(a.table + bm.d_off);
    long long* rbase = reinterpret_cast<long long*>(a.table + bm.b_off);
    long long* rzero = rbase + k;
    if (i < k) {
      const double* row = a.A + bm.a_off + (int64_t)i * k;
      double absum = 0.0;
      int fin = 1;
      for (int j = 0; j < k; ++j) {
        const double v = row[j];
        fin &= isfinite(v) ? 1 : 0;
        absum += ldexp(fabs(v), s_cexp[j]);
      }
      int kk = 0;
      if (fin && absum > 0.0) frexp(absum, &kk);
      const int s = 61 - kk;
      long long qsum = 0;
      for (int j = 0; j < k - 1; ++j) {
        const long long q = fin ? __double2ll_rn(ldexp(row[j], s - 1 + s_cexp[j])) : 0;
        qsum += 2 * q;
        RD[(2 * j) * k + i] = 4 * q;
        RD[(2 * j + 1) * k + i] = -4 * q;
      }
      const long long qn = fin ? 2 * __double2ll_rd(ldexp(row[k - 1], s - 1 + s_cexp[k - 1])) + 1 : 1;
      rbase[i] = qn - qsum;
      rzero[i] = 0;
      atomicAdd(&s_sum, s);
      atomicAdd(&s_bound, kk - 1);
      if (!fin || batch_labels_differ(a, bm, i)) atomicOr(&s_flags, 1);
      if (fin && absum == 0.0) atomicOr(&s_flags, 2);
    }
  } else if (i < k) {
    const double* row = a.A + 2 * (bm.a_off + (int64_t)i * k);
    double absum = 0.0;
    int fin = 1;
    for (int j = 0; j < 2 * k; ++j) {
      double v = row[j];
      fin &= isfinite(v) ? 1 : 0;
      absum += ldexp(fabs(v), s_cexp[j / 2]);
    }
    int kk = 0;
    if (fin && absum > 0.0) frexp(absum, &kk);
    const int s = 60 - kk;
    long long sr = 0, si = 0;
    for (int j = 0; j < k - 1; ++j) {
      long long qr = fin ? __double2ll_rn(ldexp(row[2 * j], s + s_cexp[j])) : 0;
      long long qi = fin ? __double2ll_rn(ldexp(row[2 * j + 1], s + s_cexp[j])) : 0;
      sr += qr;
      si += qi;
      D[(2 * j) * k + i] = make_longlong2(2 * qr, 2 * qi);
      D[(2 * j + 1) * k + i] = make_longlong2(-2 * qr, -2 * qi);
    }
    long long nr = fin ? __double2ll_rn(ldexp(row[2 * (k - 1)], s + s_cexp[k - 1])) : 0;
    long long ni = fin ? __double2ll_rn(ldexp(row[2 * (k - 1) + 1], s + s_cexp[k - 1])) : 0;
    base[i] = make_longlong2(nr - sr, ni - si);
    zero[i] = make_longlong2(0, 0);
    atomicAdd(&s_sum, s);
    atomicAdd(&s_bound, kk - 1);
    if (!fin || batch_labels_differ(a, bm, i)) atomicOr(&s_flags, 1);
    if (fin && absum == 0.0) atomicOr(&s_flags, 2);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    BatchMat* mm = const_cast<BatchMat*>(a.mats) + m;
    mm->sum_s = s_sum + csum;
    mm->flags = s_flags | (s_bound - csum + k > 1000 ? 4 : 0);  // the range of A itself
  }
}

// Sweep steps t in [0, 2^c) of the chunk starting at g0 of a K x K matrix
// whose table starts at D; adds the terms to (accr, acci).
template <int K>
__device__ __forceinline__ void batch_sweep(const longlong2* __restrict__ D, const longlong2* __restrict__ base,
                                            int sum_s, int c, uint64_t g0, bool active, dd& accr, dd& acci) {
  const longlong2* zero = base + K;
  const int ebase = 62 * (K + 1) - 120 - sum_s - K;
  const uint32_t nsteps = 1u << c;
  const uint32_t kb = (uint32_t)((g0 >> c) & 1u) << c;
  const uint32_t gpar = (uint32_t)(g0 & 1u);
  long long Yr[K], Yi[K];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const longlong2 b = __ldg(base + i);
    Yr[i] = b.x;
    Yi[i] = b.y;
  }
  const uint64_t G = gray64(g0);
  for (int j = (c > 0 ? c - 1 : 0); j < K - 1; ++j) {
    const long long msk = -(long long)((G >> j) & 1u);
    const longlong2* col = D + (size_t)(2 * j) * K;
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const longlong2 d = __ldg(col + i);
      Yr[i] += d.x & msk;
      Yi[i] += d.y & msk;
    }
  }
  for (uint32_t t = 0; t < nsteps; ++t) {
    const int j = __ffs(t) - 1;
    const uint32_t sb = ((t | kb) >> (j + 1)) & 1u;
    const longlong2* col = t ? D + (size_t)(2 * j + sb) * K : zero;
    CProd pa, pb;
    cprod_init(pa);
    cprod_init(pb);
    int sa = 0, sbb = 0;
#pragma unroll
    for (int i = 0; i < K; i += 2) {
      const longlong2 d0 = __ldg(col + i);
      Yr[i] += d0.x;
      Yi[i] += d0.y;
      sa += cprod_mul(pa, Yr[i], Yi[i]);
      if (i + 1 < K) {
        const longlong2 d1 = __ldg(col + i + 1);
        Yr[i + 1] += d1.x;
        Yi[i + 1] += d1.y;
        sbb += cprod_mul(pb, Yr[i + 1], Yi[i + 1]);
      }
    }
    const long long br_ = ((long long)pb.r1 << 31) | pb.r0;
    const long long bi_ = ((long long)pb.i1 << 31) | pb.i0;
    const int sm = cprod_mul(pa, br_, bi_);
    const long long zr = ((long long)pa.r1 << 31) | pa.r0;
    const long long zi = ((long long)pa.i1 << 31) | pa.i0;
    const int e = ebase - (sa + sbb + sm);
    const double hr = (double)zr, hi_ = (double)zi;
    const double lr = (double)(zr - __double2ll_rn(hr)), li = (double)(zi - __double2ll_rn(hi_));
    const double sc = ldexp(((t ^ gpar) & 1u) ? -1.0 : 1.0, e);
    dd_acc(accr, active ? hr * sc : 0.0, active ? lr * sc : 0.0);
    dd_acc(acci, active ? hi_ * sc : 0.0, active ? li * sc : 0.0);
  }
  accr = dd_make(accr.hi, accr.lo);
  acci = dd_make(acci.hi, acci.lo);
}

// The real counterpart of batch_sweep: two integer product chains as in
// ryser_real_kernel, the term split exactly into head and tail.
template <int K>
__device__ __forceinline__ void batch_sweep_real(const long long* __restrict__ D, const long long* __restrict__ base,
                                                 int sum_s, int c, uint64_t g0, bool active, dd& acc) {
  const long long* zero = base + K;
  const int K1 = 64 * K + 1025 - sum_s;
  const uint32_t nsteps = 1u << c;
  const uint32_t kb = (uint32_t)((g0 >> c) & 1u) << c;
  const uint32_t gpar = (uint32_t)(g0 & 1u);
  unsigned long long Y[K];
#pragma unroll
  for (int i = 0; i < K; ++i) Y[i] = (unsigned long long)__ldg(base + i);
  const uint64_t G = gray64(g0);
  for (int j = (c > 0 ? c - 1 : 0); j < K - 1; ++j) {
    const long long msk = -(long long)((G >> j) & 1u);
    const long long* col = D + (size_t)(2 * j) * K;
#pragma unroll
    for (int i = 0; i < K; ++i) Y[i] += (unsigned long long)(__ldg(col + i) & msk);
  }
  for (uint32_t t = 0; t < nsteps; ++t) {
    const int j = __ffs(t) - 1;
    const uint32_t sb = ((t | kb) >> (j + 1)) & 1u;
    const long long* col = t ? D + (size_t)(2 * j + sb) * K : zero;
    Prod pa, pb;
    prod_init(pa);
    prod_init(pb);
    uint32_t neg = 0, epos = 0;
#pragma unroll
    for (int i = 0; i < K; i += 2) {
      uint32_t a0, a1, ma, b0, b1, mb = 0, qb = 0;
      Y[i] += (unsigned long long)__ldg(col + i);
      row_abs(Y[i], a0, a1, ma);
      if (i + 1 < K) {
        Y[i + 1] += (unsigned long long)__ldg(col + i + 1);
        row_abs(Y[i + 1], b0, b1, mb);
      }
      const uint32_t qa = prod_mul(pa, a0, a1);
      if (i + 1 < K) qb = prod_mul(pb, b0, b1);
      neg = neg + ma + mb;
      epos = epos + qa + qb;
    }
    epos += prod_mul(pa, pb.m0, pb.m1);
    const int shifts = 30 * (K + 1) - (int)epos;
    const int f = K1 - shifts - (K + 1);
    const uint32_t signbit = (neg ^ t ^ gpar) << 31;
    double th, tl;
    prod_to_dd(pa, (uint32_t)max(f, 0), signbit, th, tl);
    dd_acc(acc, active ? th : 0.0, active ? tl : 0.0);
  }
  acc = dd_make(acc.hi, acc.lo);
}

template <int K>
__device__ __forceinline__ void batch_item_real(const BatchArgs& a, const BatchItem& it) {
  const int lane = threadIdx.x & 31;
  dd acc = {0.0, 0.0};
  const dd zero = {0.0, 0.0};
  if (it.mode == kLaneMode) {
    const bool active = lane < it.count;
    const int m = a.lane_mats[it.mat + (active ? lane : 0)];
    const BatchMat bm = a.mats[m];
    const bool ok = active && bm.flags == 0;
    if constexpr (K <= 16)  // one matrix per lane only for short sweeps (as complex)
      batch_sweep_real<K>(reinterpret_cast<const long long*>(a.table + bm.d_off),
                          reinterpret_cast<const long long*>(a.table + bm.b_off), bm.sum_s, bm.g, 0ull, ok, acc);
    if (active) {
      a.slots[2 * bm.slot0] = acc;
      a.slots[2 * bm.slot0 + 1] = zero;
    }
  } else {
    const BatchMat bm = a.mats[it.mat];
    const uint64_t chunk = (uint64_t)it.chunk0 + lane;
    const uint64_t nchunks = 1ull << (bm.g - it.c);
    const bool active = chunk < nchunks && bm.flags == 0;
    batch_sweep_real<K>(reinterpret_cast<const long long*>(a.table + bm.d_off),
                        reinterpret_cast<const long long*>(a.table + bm.b_off), bm.sum_s, it.c,
                        (active ? chunk : 0ull) << it.c, active, acc);
    acc = dd_warp_sum(acc);
    if (lane == 0) {
      a.slots[2 * it.slot] = acc;
      a.slots[2 * it.slot + 1] = zero;
    }
  }
}

// Chunked sweep of a K x K complex matrix (K >= 16) by a lane pair, as in
// ryser_cplx2_kernel: lane li of the pair holds rows li R .. li R + R - 1,
// one shuffle and one complex multiply combine the halves, each lane adds the
// terms of every second step.
template <int K>
__device__ __forceinline__ void batch_sweep2(const longlong2* __restrict__ D, const longlong2* __restrict__ base,
                                             int sum_s, int c, uint64_t g0, bool active, dd& accr, dd& acci) {
  constexpr int R = (K + 1) / 2;
  const int li = threadIdx.x & 1;
  const int eoff = -(sum_s + K) - ((K & 1) ? 60 : 0);
  const uint32_t nsteps = 1u << c;
  const uint32_t kb = (uint32_t)((g0 >> c) & 1u) << c;
  const uint32_t gpar = (uint32_t)(g0 & 1u);
  long long Yr[R], Yi[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = li * R + r;
    const longlong2 b = i < K ? __ldg(base + i) : make_longlong2(1ll << 60, 0);
    Yr[r] = b.x;
    Yi[r] = b.y;
  }
  const uint64_t G = gray64(g0);
  for (int j = (c > 0 ? c - 1 : 0); j < K - 1; ++j) {
    const long long msk = -(long long)((G >> j) & 1u);
    const longlong2* col = D + (size_t)(2 * j) * K + li * R;
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (li * R + r < K) {
        const longlong2 d = __ldg(col + r);
        Yr[r] += d.x & msk;
        Yi[r] += d.y & msk;
      }
  }
  CTerm keep = {0, 0, 0u, 0u, 0};
  uint32_t kneg = 0u;
  for (uint32_t t = 0; t < nsteps; ++t) {
    if (t) {
      const int j = __ffs(t) - 1;
      const uint32_t sb = ((t | kb) >> (j + 1)) & 1u;
      const longlong2* col = D + (size_t)(2 * j + sb) * K + li * R;
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (li * R + r < K) {
          const longlong2 d = __ldg(col + r);
          Yr[r] += d.x;
          Yi[r] += d.y;
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
    v = cterm_mul(li ? o : v, li ? v : o);
    if ((t & 1u) == (uint32_t)li) {
      keep = v;
      kneg = (t ^ gpar) & 1u;
    }
    if ((t & 1u) || t + 1 == nsteps) {
      const uint32_t tk = (t & ~1u) + (uint32_t)li;
      const bool in = active && tk <= t;
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

template <int K>
__device__ __forceinline__ void batch_item(const BatchArgs& a, const BatchItem& it) {
  const int lane = threadIdx.x & 31;
  dd accr = {0.0, 0.0}, acci = {0.0, 0.0};
  if (it.mode == kLaneMode) {
    const bool active = lane < it.count;
    const int m = a.lane_mats[it.mat + (active ? lane : 0)];
    const BatchMat bm = a.mats[m];
    const bool ok = active && bm.flags == 0;
    // one complex matrix per lane only for short sweeps (K <= 16, enforced by
    // the plan): longer rows would not fit the registers of a lane
    if constexpr (K <= 16) batch_sweep<K>(a.table + bm.d_off, a.table + bm.b_off, bm.sum_s, bm.g, 0ull, ok, accr, acci);
    if (active) {
      a.slots[2 * bm.slot0] = accr;
      a.slots[2 * bm.slot0 + 1] = acci;
    }
  } else {
    const BatchMat bm = a.mats[it.mat];
    const uint64_t chunk = (uint64_t)it.chunk0 + (K >= 16 ? (lane >> 1) : lane);
    const uint64_t nchunks = 1ull << (bm.g - it.c);
    const bool active = chunk < nchunks && bm.flags == 0;
    if constexpr (K >= 16)
      batch_sweep2<K>(a.table + bm.d_off, a.table + bm.b_off, bm.sum_s, it.c, (active ? chunk : 0ull) << it.c, active,
                      accr, acci);
    else
      batch_sweep<(K < 16 ? K : 1)>(a.table + bm.d_off, a.table + bm.b_off, bm.sum_s, it.c,
                                    (active ? chunk : 0ull) << it.c, active, accr, acci);
    accr = dd_warp_sum(accr);
    acci = dd_warp_sum(acci);
    if (lane == 0) {
      a.slots[2 * it.slot] = accr;
      a.slots[2 * it.slot + 1] = acci;
    }
  }
}

// One persistent kernel per element type (each is register-bounded for 2 CTAs
// per SM on its own).
template <bool REAL>
__global__ void __launch_bounds__(kBlock, 2) batch_main_kernel(BatchArgs a) {
  const int lane = threadIdx.x & 31;
  const uint64_t t_start = global_ns();
  for (;;) {
    // cancellation and the time budget, between work items (items left in the
    // queue stay undone; the finish kernel then marks every matrix)
    if (should_stop(a.abort_word, a.budget_ns, t_start, a.stopped)) break;
    int idx = 0;
    if (lane == 0) idx = (int)atomicAdd(a.counter, 1u);
    idx = __shfl_sync(0xffffffffu, idx, 0);
    if (idx >= a.nitems) break;
    const BatchItem it = a.items[idx];
    switch (it.k) {
#define PERM_BATCH_CASE(KK)       \
  case KK:                        \
    if constexpr (REAL)           \
      batch_item_real<KK>(a, it); \
    else                          \
      batch_item<KK>(a, it);      \
    break;
      PERM_BATCH_CASE(1) PERM_BATCH_CASE(2) PERM_BATCH_CASE(3) PERM_BATCH_CASE(4) PERM_BATCH_CASE(5)
      PERM_BATCH_CASE(6) PERM_BATCH_CASE(7) PERM_BATCH_CASE(8) PERM_BATCH_CASE(9) PERM_BATCH_CASE(10)
      PERM_BATCH_CASE(11) PERM_BATCH_CASE(12) PERM_BATCH_CASE(13) PERM_BATCH_CASE(14) PERM_BATCH_CASE(15)
      PERM_BATCH_CASE(16) PERM_BATCH_CASE(17) PERM_BATCH_CASE(18) PERM_BATCH_CASE(19) PERM_BATCH_CASE(20)
      PERM_BATCH_CASE(21) PERM_BATCH_CASE(22) PERM_BATCH_CASE(23) PERM_BATCH_CASE(24) PERM_BATCH_CASE(25)
      PERM_BATCH_CASE(26) PERM_BATCH_CASE(27) PERM_BATCH_CASE(28) PERM_BATCH_CASE(29) PERM_BATCH_CASE(30)
      PERM_BATCH_CASE(31) PERM_BATCH_CASE(32)
#undef PERM_BATCH_CASE
      default:
        break;
    }
  }
}

// v * w for a small integer weight w (exact product of the head by FMA).
__device__ __forceinline__ dd dd_scale(dd v, double w) {
  const double p = v.hi * w;
  const double e = fma(v.hi, w, -p) + v.lo * w;
  return dd_make(p, e);
}

// One thread per matrix: its slots in order (times their unit's weight),
// then the factor 2 (-1)^(k-1).
__global__ void batch_finish_kernel(BatchArgs a) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= a.nmats) return;
  const BatchOut bo = a.outs[m];
  int flags = 0;
  for (int u = bo.u0; u < bo.u0 + bo.nu; ++u) flags |= a.mats[u].flags;
  // the units of one matrix share their scales, so flags 2 (a zero row, or
  // for transposed units a zero column: perm = 0) and 4 agree between them
  dd r = {0.0, 0.0}, im = {0.0, 0.0};
  for (int s = bo.slot0; s < bo.slot0 + bo.nslots; ++s) {
    const double w = a.slot_w[s];
    const dd sr = a.slots[2 * s], si = a.slots[2 * s + 1];
    r = dd_add(r, w == 1.0 ? sr : dd_scale(sr, w));
    im = dd_add(im, w == 1.0 ? si : dd_scale(si, w));
  }
  const BatchMat bm = {bo.k, 0, flags, 0, 0, 0, 0, 0, 0, -1};
  const double f = (bm.k & 1) ? 2.0 : -2.0;
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  int32_t st = PERM_OK;
  if (bm.flags & 1) st = PERM_EINVAL;
  else if (bm.flags & 4) st = PERM_ERANGE;
  else if (*a.stopped) st = stop_status(*a.stopped);
  if (a.type == PERM_F64) {
    a.out[m] = st != PERM_OK ? nan : (bm.flags & 2) ? 0.0 : (r.hi + r.lo) * f;
  } else if (st != PERM_OK) {
    a.out[2 * m] = nan;
    a.out[2 * m + 1] = nan;
  } else if (bm.flags & 2) {
    a.out[2 * m] = 0.0;
    a.out[2 * m + 1] = 0.0;
  } else {
    a.out[2 * m] = (r.hi + r.lo) * f;
    a.out[2 * m + 1] = (im.hi + im.lo) * f;
  }
  if (a.status) a.status[m] = st;
}

}  // namespace permgpu

using namespace permgpu;

struct perm_batch_plan {
  int device = 0;
  int type = PERM_C128;
  int count = 0;
  int sms = 0;
  int max_k = 0;
  std::vector<int> ks;
  std::vector<int64_t> a_off;
  std::vector<int32_t> labels;   // row labels, sum of ks entries (empty: all rows distinct)
  std::vector<int64_t> lab_off;  // first label of every matrix
  // per size class: mode and chunk exponent
  int cls_mode[kBatchKMax + 1];
  int cls_c[kBatchKMax + 1];
  // device buffers (owned)
  BatchMat* d_mats = nullptr;
  BatchItem* d_items = nullptr;
  int32_t* d_lane_mats = nullptr;
  BatchOut* d_outs = nullptr;
  int32_t* d_desc = nullptr;
  double* d_slot_w = nullptr;
  longlong2* d_table = nullptr;
  dd* d_slots = nullptr;
  unsigned int* d_counter = nullptr;
  int nitems = 0;
  int nunits = 0;
  int nslots_total = 0;
  size_t table_elems = 0;
  // bound buffers and the captured graph
  const double* A = nullptr;
  double* out = nullptr;
  int32_t* status = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  // the graph's kernel nodes and the arguments they were last given: a replay
  // with other buffers (or a new abort word / time budget) updates them in
  // place, without a new capture or any allocation
  std::vector<cudaGraphNode_t> knodes;
  BatchArgs bound_args;
};

static void batch_free(perm_batch_plan* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  cudaFree(p->d_mats);
  cudaFree(p->d_items);
  cudaFree(p->d_lane_mats);
  cudaFree(p->d_outs);
  cudaFree(p->d_desc);
  cudaFree(p->d_slot_w);
  cudaFree(p->d_table);
  cudaFree(p->d_slots);
  cudaFree(p->d_counter);
  delete p;
}

// Default choice per size class: one matrix per lane while a sweep is short,
// otherwise chunks of 2^c steps with at least ~8 warp items per matrix, and
// c <= 12: a warp item is then at most 2^17 steps, a few ms of one warp, so
// the last wave of the queue stays short (with c = k - 9 a k = 26 item ran
// for about 0.4 s, and how full its last wave was decided the run time).
static void batch_default_classes(perm_batch_plan* p) {
  for (int k = 0; k <= kBatchKMax; ++k) {
    if (k <= 14) {
      p->cls_mode[k] = kLaneMode;
      p->cls_c[k] = k > 0 ? k - 1 : 0;
    } else {
      p->cls_mode[k] = kWarpMode;
      int c = k - 1 - 5 - 3;  // 32 chunks per item, 8 items per matrix
      if (c > 12) c = 12;
      if (c < 6) c = 6;
      if (c > k - 1) c = k - 1;
      p->cls_c[k] = c;
    }
  }
}

// Sweep units of one matrix.  Without repeated labels: the matrix itself
// (g = k - 1, weight 1).  With them: the transposed sweeps of the grouped
// Glynn sum (see the top of this file), when they have fewer terms.
struct UnitPlan {
  int g;
  double w;
  std::vector<int32_t> desc;  // empty: plain
  std::vector<int32_t> chk;   // empty, or P, (a, b) x P: labelled rows that must be equal
};

static void plan_units_for(int k, const int32_t* labels, std::vector<UnitPlan>& units) {
  units.clear();
  UnitPlan plain{k - 1, 1.0, {}, {}};
  if (!labels || k < 2) {
    units.push_back(plain);
    return;
  }
  // groups of equal labels, in order of first appearance
  std::vector<int32_t> lab(labels, labels + k);
  std::vector<std::vector<int>> groups;
  for (int r = 0; r < k; ++r) {
    size_t gi = 0;
    while (gi < groups.size() && lab[groups[gi][0]] != lab[r]) ++gi;
    if (gi == groups.size()) groups.emplace_back();
    groups[gi].push_back(r);
  }
  if ((int)groups.size() == k) {
    units.push_back(plain);
    return;
  }
  std::vector<int32_t> chk(1, 0);
  for (const auto& gr : groups)
    for (size_t t = 1; t < gr.size(); ++t) {
      chk.push_back(gr[0]);
      chk.push_back(gr[t]);
      chk[0]++;
    }
  plain.chk = chk;
  // fix one copy of a singleton row if there is one, else of the smallest group
  size_t fx = 0;
  for (size_t gi = 0; gi < groups.size(); ++gi)
    if (groups[gi].size() < groups[fx].size()) fx = gi;
  std::vector<int> tog;
  std::vector<std::pair<int, int>> repd;  // (row, multiplicity)
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    const int mu = (int)groups[gi].size() - (gi == fx ? 1 : 0);
    const int r0 = groups[gi][0];
    if (mu == 1) tog.push_back(r0);
    else if (mu >= 2) repd.push_back({r0, mu});
  }
  // at most kMaxUnits combinations, each a sweep of at least 2^min(k-1, 8)
  // steps: expand repeated groups back into Gray bits (smallest first: a
  // pair costs 4/3 of its terms) until both hold
  constexpr int kMaxUnits = 64;
  const int gmin = std::min(k - 1, 8);
  double combos = 1.0;
  for (auto& rm : repd) combos *= rm.second + 1;
  while ((combos > kMaxUnits || (int)tog.size() < gmin) && !repd.empty()) {
    size_t sm = 0;
    for (size_t t = 1; t < repd.size(); ++t)
      if (repd[t].second < repd[sm].second) sm = t;
    for (int q = 0; q < repd[sm].second; ++q) tog.push_back(repd[sm].first);
    combos /= repd[sm].second + 1;
    repd.erase(repd.begin() + sm);
  }
  const int G = (int)tog.size();
  if (std::ldexp(combos, G) >= std::ldexp(1.0, k - 1)) {
    units.push_back(plain);
    return;
  }
  // every combination (k_rho) of the repeated rows: coefficient mu - 2 k_rho,
  // weight prod C(mu, k_rho) (-1)^(k_rho); times (-1)^(G - (k-1)) for the
  // sign of the toggled rows against the plain sweep's 2 (-1)^(k-1)
  std::vector<int> kr(repd.size(), 0);
  for (bool first = true;; first = false) {
    UnitPlan u;
    u.g = G;
    double w = ((G - (k - 1)) & 1) ? -1.0 : 1.0;
    u.desc.push_back(groups[fx][0]);
    u.desc.push_back(G);
    for (int t : tog) u.desc.push_back(t);
    u.desc.push_back((int32_t)repd.size());
    for (size_t t = 0; t < repd.size(); ++t) {
      const int mu = repd[t].second;
      u.desc.push_back(repd[t].first);
      u.desc.push_back(mu - 2 * kr[t]);
      double c = 1.0;
      for (int q = 0; q < kr[t]; ++q) c = c * (mu - q) / (q + 1);
      w *= (kr[t] & 1) ? -c : c;
    }
    if (first) u.chk = chk;  // equality checks once per matrix
    u.w = w;
    units.push_back(std::move(u));
    size_t t = 0;
    while (t < repd.size() && ++kr[t] > repd[t].second) kr[t++] = 0;
    if (t == repd.size()) break;
  }
}

static void plan_units(const perm_batch_plan* p, int m, std::vector<UnitPlan>& units) {
  plan_units_for(p->ks[m], p->labels.empty() ? nullptr : p->labels.data() + p->lab_off[m], units);
}

// Build the sweep units, work queue, slots and records for the current class
// choices (host), and upload them.
static int batch_build(perm_batch_plan* p) {
  struct Unit {
    int m, g, combo;
    double w;
    std::vector<int32_t> desc, chk;
  };
  std::vector<Unit> all;
  std::vector<UnitPlan> ups;
  for (int m = 0; m < p->count; ++m) {
    plan_units(p, m, ups);
    for (size_t c = 0; c < ups.size(); ++c)
      all.push_back({m, ups[c].g, (int)c, ups[c].w, std::move(ups[c].desc), std::move(ups[c].chk)});
  }
  // units of one size and Gray length together, then by matrix: the units
  // (and slots) of every matrix are contiguous
  std::stable_sort(all.begin(), all.end(), [&](const Unit& x, const Unit& y) {
    const int kx = p->ks[x.m], ky = p->ks[y.m];
    if (kx != ky) return kx < ky;
    if (x.g != y.g) return x.g < y.g;
    return x.m < y.m;
  });
  const int nu = (int)all.size();
  // D of every matrix (plain ones followed by their base and zero vectors),
  // then base and zero of every transposed unit; in longlong2 units (a real
  // table holds two int64 per longlong2)
  const bool realt = p->type == PERM_F64;
  auto d_size = [&](int k) -> int64_t { return (int64_t)(realt ? 1 : 2) * (k > 1 ? k - 1 : 0) * k; };
  auto b_size = [&](int k) -> int64_t { return (int64_t)(realt ? 1 : 2) * k; };
  std::vector<int64_t> dm(p->count);
  std::vector<char> transposed(p->count, 0);
  for (const Unit& un : all)
    if (!un.desc.empty()) transposed[un.m] = 1;
  size_t toff = 0;
  for (int m = 0; m < p->count; ++m) {
    dm[m] = (int64_t)toff;
    toff += d_size(p->ks[m]) + (transposed[m] ? 0 : b_size(p->ks[m]));
  }
  std::vector<BatchMat> mats(nu);
  std::vector<BatchOut> outs(p->count);
  std::vector<int32_t> desc;
  std::vector<double> slot_w;
  std::vector<BatchItem> items;
  std::vector<int32_t> lane_mats;
  for (int u = 0; u < nu; ++u) {
    const int m = all[u].m, k = p->ks[m];
    mats[u].k = k;
    mats[u].sum_s = 0;
    mats[u].flags = 0;
    mats[u].a_off = p->a_off[m];
    mats[u].d_off = dm[m];
    if (transposed[m]) {
      mats[u].b_off = (int64_t)toff;
      toff += b_size(k);
    } else {
      mats[u].b_off = dm[m] + d_size(k);
    }
    mats[u].g = all[u].g;
    mats[u].desc = all[u].desc.empty() ? -1 : (int32_t)desc.size();
    desc.insert(desc.end(), all[u].desc.begin(), all[u].desc.end());
    mats[u].chk = all[u].chk.empty() ? -1 : (int32_t)desc.size();
    desc.insert(desc.end(), all[u].chk.begin(), all[u].chk.end());
  }
  p->table_elems = toff;
  p->nunits = nu;
  // slots: lane-mode units one slot, warp-mode one per item
  int slot = 0;
  auto add_slot = [&](int u) {
    slot_w.push_back(all[u].w);
    return slot++;
  };
  for (int u0 = 0; u0 < nu;) {
    const int k = p->ks[all[u0].m], g = all[u0].g;
    int u1 = u0;
    while (u1 < nu && p->ks[all[u1].m] == k && all[u1].g == g) ++u1;
    if (p->cls_mode[k] == kLaneMode) {
      for (int q0 = u0; q0 < u1; q0 += 32) {
        BatchItem it;
        memset(&it, 0, sizeof(it));
        it.mode = kLaneMode;
        it.k = k;
        it.c = g;
        it.count = std::min(32, u1 - q0);
        it.mat = (int)lane_mats.size();
        for (int q = 0; q < it.count; ++q) {
          lane_mats.push_back(q0 + q);
          mats[q0 + q].slot0 = add_slot(q0 + q);
        }
        items.push_back(it);
      }
    } else {
      const int c = std::min(p->cls_c[k], g);
      const uint64_t nchunks = 1ull << (g - c);
      // complex k >= 16: lane pairs, 16 chunks per warp item
      const uint64_t per_item = (p->type == PERM_C128 && k >= 16) ? 16 : 32;
      for (int u = u0; u < u1; ++u) {
        mats[u].slot0 = slot;
        for (uint64_t ch = 0; ch < nchunks; ch += per_item) {
          BatchItem it;
          memset(&it, 0, sizeof(it));
          it.mode = kWarpMode;
          it.k = k;
          it.c = c;
          it.count = (int)per_item;
          it.mat = u;
          it.slot = add_slot(u);
          it.chunk0 = (int64_t)ch;
          items.push_back(it);
        }
      }
    }
    u0 = u1;
  }
  // output records: first unit, unit count and slot range of every matrix
  for (int m = 0; m < p->count; ++m) outs[m] = {p->ks[m], -1, 0, 0, 0, 0};
  for (int u = 0; u < nu; ++u) {
    BatchOut& o = outs[all[u].m];
    if (o.u0 < 0) {
      o.u0 = u;
      o.slot0 = mats[u].slot0;
    }
    o.nu++;
  }
  for (int m = 0; m < p->count; ++m) {
    const BatchOut& o = outs[m];
    const int ulast = o.u0 + o.nu - 1;
    int end = ulast + 1 < nu ? mats[ulast + 1].slot0 : slot;
    outs[m].nslots = end - o.slot0;
  }
  // longest first: cost ~ steps x k per item
  std::vector<size_t> idx(items.size());
  for (size_t i = 0; i < idx.size(); ++i) idx[i] = i;
  auto cost = [&](const BatchItem& it) {
    double steps = (double)(1ull << it.c);
    return steps * (it.k + 4);
  };
  std::stable_sort(idx.begin(), idx.end(), [&](size_t x, size_t y) { return cost(items[x]) > cost(items[y]); });
  std::vector<BatchItem> sorted(items.size());
  for (size_t i = 0; i < idx.size(); ++i) sorted[i] = items[idx[i]];
  p->nitems = (int)sorted.size();
  p->nslots_total = slot;

  cudaFree(p->d_mats);
  cudaFree(p->d_items);
  cudaFree(p->d_lane_mats);
  cudaFree(p->d_outs);
  cudaFree(p->d_desc);
  cudaFree(p->d_slot_w);
  cudaFree(p->d_table);
  cudaFree(p->d_slots);
  p->d_mats = nullptr;
  p->d_items = nullptr;
  p->d_lane_mats = nullptr;
  p->d_outs = nullptr;
  p->d_desc = nullptr;
  p->d_slot_w = nullptr;
  p->d_table = nullptr;
  p->d_slots = nullptr;
  if (cudaMalloc(&p->d_mats, sizeof(BatchMat) * std::max(1, nu)) != cudaSuccess ||
      cudaMalloc(&p->d_items, sizeof(BatchItem) * std::max(1, p->nitems)) != cudaSuccess ||
      cudaMalloc(&p->d_lane_mats, sizeof(int32_t) * std::max<size_t>(1, lane_mats.size())) != cudaSuccess ||
      cudaMalloc(&p->d_outs, sizeof(BatchOut) * std::max(1, p->count)) != cudaSuccess ||
      cudaMalloc(&p->d_desc, sizeof(int32_t) * std::max<size_t>(1, desc.size())) != cudaSuccess ||
      cudaMalloc(&p->d_slot_w, sizeof(double) * std::max(1, p->nslots_total)) != cudaSuccess ||
      cudaMalloc(&p->d_table, sizeof(longlong2) * std::max<size_t>(1, p->table_elems)) != cudaSuccess ||
      cudaMalloc(&p->d_slots, sizeof(dd) * 2 * std::max(1, p->nslots_total)) != cudaSuccess) {
    cudaGetLastError();
    return PERM_ENOMEM;
  }
  if (!p->d_counter && cudaMalloc(&p->d_counter, 2 * sizeof(unsigned int)) != cudaSuccess) {
    cudaGetLastError();
    return PERM_ENOMEM;
  }
  if (cudaMemcpy(p->d_mats, mats.data(), sizeof(BatchMat) * nu, cudaMemcpyHostToDevice) != cudaSuccess ||
      (p->nitems && cudaMemcpy(p->d_items, sorted.data(), sizeof(BatchItem) * p->nitems, cudaMemcpyHostToDevice) !=
                        cudaSuccess) ||
      (!lane_mats.empty() && cudaMemcpy(p->d_lane_mats, lane_mats.data(), sizeof(int32_t) * lane_mats.size(),
                                        cudaMemcpyHostToDevice) != cudaSuccess) ||
      cudaMemcpy(p->d_outs, outs.data(), sizeof(BatchOut) * p->count, cudaMemcpyHostToDevice) != cudaSuccess ||
      (!desc.empty() && cudaMemcpy(p->d_desc, desc.data(), sizeof(int32_t) * desc.size(), cudaMemcpyHostToDevice) !=
                            cudaSuccess) ||
      cudaMemcpy(p->d_slot_w, slot_w.data(), sizeof(double) * p->nslots_total, cudaMemcpyHostToDevice) != cudaSuccess)
    return PERM_ECUDA;
  return PERM_OK;
}

static BatchArgs batch_args(const perm_batch_plan* p) {
  BatchArgs a;
  memset(&a, 0, sizeof(a));
  a.A = p->A;
  a.mats = p->d_mats;
  a.outs = p->d_outs;
  a.desc = p->d_desc;
  a.slot_w = p->d_slot_w;
  a.items = p->d_items;
  a.lane_mats = p->d_lane_mats;
  a.table = p->d_table;
  a.slots = p->d_slots;
  a.counter = p->d_counter;
  a.out = p->out;
  a.status = p->status;
  a.abort_word = current_abort_word();
  a.stopped = p->d_counter + 1;
  a.budget_ns = current_time_budget();
  a.nmats = p->count;
  a.nunits = p->nunits;
  a.nitems = p->nitems;
  a.type = p->type;
  return a;
}

// The execution sequence (captured into the plan's graph).
static int batch_enqueue(const perm_batch_plan* p, cudaStream_t s) {
  BatchArgs a = batch_args(p);
  if (cudaMemsetAsync(p->d_counter, 0, 2 * sizeof(unsigned int), s) != cudaSuccess) return PERM_ECUDA;
  batch_prep_kernel<<<p->nunits, kBlock, 0, s>>>(a);
  int nb = 0;
  const bool real = p->type == PERM_F64;
  const void* mk = real ? reinterpret_cast<const void*>(batch_main_kernel<true>)
                        : reinterpret_cast<const void*>(batch_main_kernel<false>);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, mk, kBlock, 0) != cudaSuccess || nb < 1) nb = 1;
  int want = (p->nitems + kWarps - 1) / kWarps;
  int grid = std::max(1, std::min(p->sms * nb, want));
  if (real)
    batch_main_kernel<true><<<grid, kBlock, 0, s>>>(a);
  else
    batch_main_kernel<false><<<grid, kBlock, 0, s>>>(a);
  batch_finish_kernel<<<(p->count + 127) / 128, 128, 0, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? PERM_OK : PERM_ECUDA;
}

static int batch_capture(perm_batch_plan* p) {
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  p->exec = nullptr;
  p->graph = nullptr;
  cudaStream_t cs;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return PERM_ECUDA;
  int rc = PERM_OK;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = PERM_ECUDA;
  if (!rc) rc = batch_enqueue(p, cs);
  cudaGraph_t g = nullptr;
  if (cudaStreamEndCapture(cs, &g) != cudaSuccess) rc = PERM_ECUDA;
  if (!rc && cudaGraphInstantiate(&p->exec, g, 0) != cudaSuccess) rc = PERM_ECUDA;
  p->graph = g;
  cudaStreamDestroy(cs);
  p->knodes.clear();
  if (!rc) {
    size_t num = 0;
    if (cudaGraphGetNodes(g, nullptr, &num) != cudaSuccess) rc = PERM_ECUDA;
    std::vector<cudaGraphNode_t> nodes(num);
    if (!rc && num && cudaGraphGetNodes(g, nodes.data(), &num) != cudaSuccess) rc = PERM_ECUDA;
    for (size_t i = 0; i < num && !rc; ++i) {
      cudaGraphNodeType t;
      if (cudaGraphNodeGetType(nodes[i], &t) != cudaSuccess) rc = PERM_ECUDA;
      else if (t == cudaGraphNodeTypeKernel) p->knodes.push_back(nodes[i]);
    }
    p->bound_args = batch_args(p);
  }
  if (rc) cudaGetLastError();
  return rc;
}

static bool same_args(const BatchArgs& x, const BatchArgs& y) {
  return x.A == y.A && x.out == y.out && x.status == y.status && x.abort_word == y.abort_word &&
         x.budget_ns == y.budget_ns;
}

// Point the instantiated graph's kernels at new buffers (every kernel of the
// plan takes the one BatchArgs block).  No allocation, no capture.
static int batch_rebind(perm_batch_plan* p, const BatchArgs& a) {
  for (cudaGraphNode_t nd : p->knodes) {
    cudaKernelNodeParams kp;
    if (cudaGraphKernelNodeGetParams(nd, &kp) != cudaSuccess) return PERM_ECUDA;
    BatchArgs arg = a;
    void* params[] = {&arg};
    kp.kernelParams = params;
    kp.extra = nullptr;
    if (cudaGraphExecKernelNodeSetParams(p->exec, nd, &kp) != cudaSuccess) {
      cudaGetLastError();
      return PERM_ECUDA;
    }
  }
  p->bound_args = a;
  return PERM_OK;
}

static int batch_create(perm_batch_plan** plan, int type, const int* ns_host, int count, const void* A_packed,
                        const int64_t* offsets_host, void* out, int32_t* status, const int32_t* labels_host) {
  if (!plan) return PERM_EINVAL;
  *plan = nullptr;
  if (type != PERM_C128 && type != PERM_F64) return PERM_EINVAL;
  if (count < 1 || !ns_host || !offsets_host || !A_packed || !out) return PERM_EINVAL;
  perm_batch_plan* p = new perm_batch_plan();
  p->type = type;
  if (cudaGetDevice(&p->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) {
    delete p;
    return PERM_ECUDA;
  }
  p->count = count;
  p->ks.assign(ns_host, ns_host + count);
  p->a_off.assign(offsets_host, offsets_host + count);
  for (int k : p->ks) {
    if (k < 1 || k > kBatchKMax) {
      delete p;
      return PERM_ERANGE;
    }
    p->max_k = std::max(p->max_k, k);
  }
  for (int64_t o : p->a_off)
    if (o < 0) {
      delete p;
      return PERM_EINVAL;
    }
  if (labels_host) {
    int64_t tot = 0;
    for (int k : p->ks) {
      p->lab_off.push_back(tot);
      tot += k;
    }
    p->labels.assign(labels_host, labels_host + tot);
  }
  p->A = static_cast<const double*>(A_packed);
  p->out = static_cast<double*>(out);
  p->status = status;
  batch_default_classes(p);
  int rc = batch_build(p);
  if (!rc) rc = batch_capture(p);
  if (rc) {
    batch_free(p);
    return rc;
  }
  *plan = p;
  return PERM_OK;
}

extern "C" int perm_batched_plan_create(perm_batch_plan** plan, int type, const int* ns_host, int count,
                                        const void* A_packed, const int64_t* offsets_host, void* out,
                                        int32_t* status) {
  return batch_create(plan, type, ns_host, count, A_packed, offsets_host, out, status, nullptr);
}

extern "C" int perm_batched_plan_create_labeled(perm_batch_plan** plan, int type, const int* ns_host, int count,
                                                const void* A_packed, const int64_t* offsets_host, void* out,
                                                int32_t* status, const int32_t* row_labels_host) {
  if (!row_labels_host) {
    if (plan) *plan = nullptr;
    return PERM_EINVAL;
  }
  return batch_create(plan, type, ns_host, count, A_packed, offsets_host, out, status, row_labels_host);
}

extern "C" int perm_batched_units(int k, const int32_t* labels, int max_units, int32_t* gray_bits, double* weight,
                                  int32_t* desc, int desc_cap, int32_t* desc_off) {
  if (k < 1 || k > kBatchKMax) return -PERM_ERANGE;
  if (max_units < 0 || desc_cap < 0) return -PERM_EINVAL;
  std::vector<UnitPlan> ups;
  plan_units_for(k, labels, ups);
  int pos = 0;
  for (size_t u = 0; u < ups.size() && (int)u < max_units; ++u) {
    if (gray_bits) gray_bits[u] = ups[u].g;
    if (weight) weight[u] = ups[u].w;
    if (desc_off) desc_off[u] = ups[u].desc.empty() ? -1 : pos;
    if (!ups[u].desc.empty()) {
      if (pos + (int)ups[u].desc.size() > desc_cap) return -PERM_ENOMEM;
      if (desc) std::copy(ups[u].desc.begin(), ups[u].desc.end(), desc + pos);
      pos += (int)ups[u].desc.size();
    }
  }
  return (int)ups.size();
}

extern "C" int perm_batched(perm_batch_plan* plan, const void* A_packed, void* out, int32_t* status, void* stream) {
  if (!plan || !plan->exec) return PERM_EINVAL;
  BatchArgs a = batch_args(plan);
  if (A_packed) a.A = static_cast<const double*>(A_packed);
  if (out) a.out = static_cast<double*>(out);
  if (status) a.status = status;
  if (!same_args(a, plan->bound_args)) {
    int rc = batch_rebind(plan, a);
    if (rc) return rc;
  }
  return cudaGraphLaunch(plan->exec, static_cast<cudaStream_t>(stream)) == cudaSuccess ? PERM_OK : PERM_ECUDA;
}

extern "C" int perm_batched_autotune(perm_batch_plan* plan, int rounds, void* stream) {
  if (!plan) return PERM_EINVAL;
  if (rounds < 1) rounds = 1;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return PERM_ECUDA;
  // tune one size class at a time: plans that hold only that class's matrices
  int rc = PERM_OK;
  for (int k = 1; k <= kBatchKMax && !rc; ++k) {
    std::vector<int> ks;
    std::vector<int64_t> offs, loffs;
    std::vector<int32_t> labs;
    for (int m = 0; m < plan->count; ++m)
      if (plan->ks[m] == k) {
        ks.push_back(k);
        offs.push_back(plan->a_off[m]);
        if (!plan->labels.empty()) {
          loffs.push_back((int64_t)labs.size());
          labs.insert(labs.end(), plan->labels.begin() + plan->lab_off[m], plan->labels.begin() + plan->lab_off[m] + k);
        }
      }
    if (ks.empty()) continue;
    struct Cand {
      int mode, c;
    };
    std::vector<Cand> cands;
    if (k <= 16) cands.push_back({kLaneMode, k - 1});
    for (int c = std::max(2, k - 1 - 12); c <= k - 1 - 5; ++c) cands.push_back({kWarpMode, c});
    if (cands.empty()) cands.push_back({k <= 16 ? kLaneMode : kWarpMode, k <= 16 ? k - 1 : std::max(0, k - 6)});
    float best = 1e30f;
    Cand pick = {plan->cls_mode[k], plan->cls_c[k]};
    for (const Cand& cd : cands) {
      perm_batch_plan* q = new perm_batch_plan();
      q->type = plan->type;
      q->device = plan->device;
      q->sms = plan->sms;
      q->count = (int)ks.size();
      q->ks = ks;
      q->a_off = offs;
      q->labels = labs;
      q->lab_off = loffs;
      q->max_k = k;
      q->A = plan->A;
      q->out = plan->out;  // scratch use of the caller's output (rewritten below)
      q->status = nullptr;
      batch_default_classes(q);
      q->cls_mode[k] = cd.mode;
      q->cls_c[k] = cd.c;
      int r = batch_build(q);
      float ms = 1e30f;
      if (!r) {
        batch_enqueue(q, s);  // warm-up
        cudaEventRecord(e0, s);
        for (int it = 0; it < rounds; ++it) batch_enqueue(q, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
      }
      batch_free(q);
      if (ms < best) {
        best = ms;
        pick = cd;
      }
    }
    plan->cls_mode[k] = pick.mode;
    plan->cls_c[k] = pick.c;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!rc) rc = batch_build(plan);
  if (!rc) rc = batch_capture(plan);
  return rc;
}

extern "C" int perm_batched_plan_info(const perm_batch_plan* plan, int k, int* mode, int* c, int* nitems) {
  if (!plan || k < 0 || k > kBatchKMax) return PERM_EINVAL;
  if (mode) *mode = plan->cls_mode[k];
  if (c) *c = plan->cls_c[k];
  if (nitems) *nitems = plan->nitems;
  return PERM_OK;
}

extern "C" void perm_batched_plan_destroy(perm_batch_plan* plan) { batch_free(plan); }
