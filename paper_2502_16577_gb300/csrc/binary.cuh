// Exact 0/1 Ryser kernel (Alg. 1 in Nijenhuis-Wilf form, chunked as Alg. 3
// with power-of-two chunks, Sec. 3.1.1) in wrap-around integer arithmetic.
//
// With the doubled rows x'_i = 2 x_i = 2 a_{i,n-1} - r_i + 2 sum_{j in S} a_ij
// every quantity is an integer: |x'_i| <= r_i <= n, the sum over the whole
// sweep is (-1)^(n-1) 2^(n-1) perm(A), and it is accumulated modulo 2^(32L)
// (L = 5 or 6 limbs).  Reduction modulo 2^W is a ring homomorphism, so
// overflow of intermediate products and sums is harmless; the result is
// perm(A) mod 2^(W-n+1), which is perm(A) itself whenever Bregman's bound
// prod_i (r_i!)^(1/r_i) is below 2^(W-n+1).
//
// Per step: one int32 add per row, signed products of five rows in int32
// (|product| < 63^5 < 2^31), then the magnitudes of the group products are
// multiplied in a limb tree and the signed term is added to the W-bit
// accumulator.  The limb tree runs on the IMAD pipe, the adds on the ALU pipe.
#pragma once

#include "common.cuh"

namespace permgpu {

template <int L>
struct Big {
  uint32_t w[L];
};

// r = a * b mod 2^(32 R), a of LA limbs, b of LB limbs (operand scanning;
// every partial sum a_i b_j + r + carry < 2^64).
template <int R, int LA, int LB>
__device__ __forceinline__ void big_mul(uint32_t (&r)[R], const uint32_t (&a)[LA], const uint32_t (&b)[LB]) {
#pragma unroll
  for (int k = 0; k < R; ++k) r[k] = 0u;
#pragma unroll
  for (int i = 0; i < LA; ++i) {
    if (i >= R) break;
    uint32_t carry = 0u;
#pragma unroll
    for (int j = 0; j < LB; ++j) {
      if (i + j >= R) break;
      unsigned long long t = (unsigned long long)a[i] * b[j] + r[i + j] + carry;
      r[i + j] = (uint32_t)t;
      carry = (uint32_t)(t >> 32);
    }
    if (i + LB < R) r[i + LB] = carry;
  }
}

// acc += (neg ? -v : v) modulo 2^(32 L), v given by LV <= L limbs.
template <int L, int LV>
__device__ __forceinline__ void big_acc_signed(uint32_t (&acc)[L], const uint32_t (&v)[LV], uint32_t negmask) {
  // acc + (v xor m) + (m & 1): two's complement negation folded into the add
  unsigned long long c = negmask & 1u;
#pragma unroll
  for (int k = 0; k < L; ++k) {
    uint32_t vk = (k < LV ? v[k] : 0u) ^ negmask;
    unsigned long long t = (unsigned long long)acc[k] + vk + c;
    acc[k] = (uint32_t)t;
    c = t >> 32;
  }
}

template <int N>
struct BinLayout {
  static constexpr int NP = (N + 3) & ~3;  // rows padded to 4: 16-byte loads
  static constexpr int NCOL = N > 1 ? N - 1 : 0;
  static constexpr size_t kD = 0;
  static constexpr size_t kBase = kD + sizeof(int32_t) * 2 * NCOL * NP;
  static constexpr size_t kZero = kBase + sizeof(int32_t) * NP;
  static constexpr size_t kBytes = kZero + sizeof(int32_t) * NP;
};

struct BinShared {
  int bad_entry;
  int zero_row;
  float bound_log2;  // log2 of Bregman's bound prod_i (r_i!)^(1/r_i)
};

template <int N>
__device__ __forceinline__ void bin_stage(const uint8_t* __restrict__ A, unsigned char* smem, BinShared& sh) {
  using Lo = BinLayout<N>;
  int32_t* D = reinterpret_cast<int32_t*>(smem + Lo::kD);
  int32_t* base = reinterpret_cast<int32_t*>(smem + Lo::kBase);
  int32_t* zero = reinterpret_cast<int32_t*>(smem + Lo::kZero);
  if (threadIdx.x == 0) {
    sh.bad_entry = 0;
    sh.zero_row = 0;
    sh.bound_log2 = 0.0f;
  }
  __syncthreads();
  int i = threadIdx.x;
  if (i < N) {
    const uint8_t* row = A + (size_t)i * N;
    int r = 0, bad = 0;
    for (int j = 0; j < N; ++j) {
      uint8_t v = row[j];
      bad |= v > 1u;
      r += v & 1u;
    }
    for (int j = 0; j < N - 1; ++j) {
      int32_t d = 2 * (int32_t)(row[j] & 1u);
      D[(2 * j) * Lo::NP + i] = d;
      D[(2 * j + 1) * Lo::NP + i] = -d;
    }
    base[i] = 2 * (int32_t)(row[N - 1] & 1u) - r;
    zero[i] = 0;
    if (bad) atomicOr(&sh.bad_entry, 1);
    if (r == 0) atomicOr(&sh.zero_row, 1);
    // log2((r!)^(1/r)) with a small upward margin
    if (r > 0) atomicAdd(&sh.bound_log2, (float)(lgamma((double)r + 1.0) / ((double)r * 0.6931471805599453)) + 1e-4f);
  } else if (i < Lo::NP) {
    for (int j = 0; j < N - 1; ++j) {
      D[(2 * j) * Lo::NP + i] = 0;
      D[(2 * j + 1) * Lo::NP + i] = 0;
    }
    base[i] = 1;  // padding rows contribute a factor 1
    zero[i] = 0;
  }
  __syncthreads();
}

// |term| of one step as an R-limb number and its sign mask, from the rows x.
template <int N, int R>
__device__ __forceinline__ void bin_term(const int32_t (&x)[N], uint32_t (&mag)[R], uint32_t& negmask) {
  constexpr int G = (N + 4) / 5;       // groups of five rows
  constexpr int P = (G + 1) / 2;       // pair products (64-bit)
  uint32_t par = 0u;
  uint32_t gm[G];
#pragma unroll
  for (int k = 0; k < G; ++k) {
    int32_t g = x[5 * k];
#pragma unroll
    for (int q = 1; q < 5; ++q)
      if (5 * k + q < N) g *= x[5 * k + q];
    par ^= (uint32_t)g;
    gm[k] = (uint32_t)(g < 0 ? -g : g);
  }
  negmask = (uint32_t)((int32_t)par >> 31);
  // level 1: pairs of groups -> 64-bit
  uint32_t p[P][2];
#pragma unroll
  for (int k = 0; k < P; ++k) {
    unsigned long long t = (unsigned long long)gm[2 * k] * (2 * k + 1 < G ? gm[2 * k + 1] : 1u);
    p[k][0] = (uint32_t)t;
    p[k][1] = (uint32_t)(t >> 32);
  }
  // level 2 and up: multiply the 64-bit pieces into the R-limb magnitude
  uint32_t acc[R];
#pragma unroll
  for (int k = 0; k < R; ++k) acc[k] = 0u;
  acc[0] = p[0][0];
  if (R > 1) acc[1] = p[0][1];
#pragma unroll
  for (int k = 1; k < P; ++k) {
    uint32_t t[R];
    big_mul<R, R, 2>(t, acc, p[k]);
#pragma unroll
    for (int q = 0; q < R; ++q) acc[q] = t[q];
  }
#pragma unroll
  for (int q = 0; q < R; ++q) mag[q] = acc[q];
}

template <int N, int L>
__global__ void __launch_bounds__(kBlock, 2) ryser_bin_kernel(RyserArgs a) {
  using Lo = BinLayout<N>;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ BinShared sh;
  bin_stage<N>(static_cast<const uint8_t*>(a.A), smem, sh);
  const int32_t* D = reinterpret_cast<const int32_t*>(smem + Lo::kD);
  const int32_t* base = reinterpret_cast<const int32_t*>(smem + Lo::kBase);
  const int32_t* zero = reinterpret_cast<const int32_t*>(smem + Lo::kZero);
  const bool skip = sh.bad_entry || sh.zero_row;

  uint32_t acc[L];
#pragma unroll
  for (int k = 0; k < L; ++k) acc[k] = 0u;
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

    int32_t x[N];
#pragma unroll
    for (int i = 0; i < N; ++i) x[i] = base[i];
    const uint64_t G = gray64(g0);
    for (int j = (a.c > 0 ? a.c - 1 : 0); j < N - 1; ++j) {
      const int32_t msk = -(int32_t)((G >> j) & 1u);
      const int32_t* col = D + (size_t)(2 * j) * Lo::NP;
#pragma unroll
      for (int i = 0; i < N; ++i) x[i] += col[i] & msk;
    }

    for (uint32_t t = 0; t < nsteps; ++t) {
      const int j = __ffs(t) - 1;
      const uint32_t sb = ((t | kb) >> (j + 1)) & 1u;
      const int4* col = reinterpret_cast<const int4*>(t ? D + (size_t)(2 * j + sb) * Lo::NP : zero);
#pragma unroll
      for (int p = 0; p < Lo::NP / 4; ++p) {
        const int4 d = col[p];
        if (4 * p + 0 < N) x[4 * p + 0] += d.x;
        if (4 * p + 1 < N) x[4 * p + 1] += d.y;
        if (4 * p + 2 < N) x[4 * p + 2] += d.z;
        if (4 * p + 3 < N) x[4 * p + 3] += d.w;
      }
      uint32_t mag[L], negmask;
      bin_term<N, L>(x, mag, negmask);
      negmask ^= (uint32_t)(-(int32_t)((t ^ gpar) & 1u));  // (-1)^g
      if (t - tlo < tcnt) big_acc_signed<L, L>(acc, mag, negmask);
    }
  }

  // reduction: sum of the lanes' W-bit residues (exact, order-free)
  __shared__ uint32_t s_acc[kWarps][L];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    uint32_t o[L];
#pragma unroll
    for (int q = 0; q < L; ++q) o[q] = __shfl_down_sync(0xffffffffu, acc[q], off);
    big_acc_signed<L, L>(acc, o, 0u);
  }
  const int w = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < L; ++q) s_acc[w][q] = acc[q];
  __syncthreads();
  uint32_t* part = static_cast<uint32_t*>(a.part);  // 8 words per CTA
  if (threadIdx.x == 0) {
    uint32_t b[L];
#pragma unroll
    for (int q = 0; q < L; ++q) b[q] = 0u;
    for (int ww = 0; ww < kWarps; ++ww) {
      uint32_t o[L];
#pragma unroll
      for (int q = 0; q < L; ++q) o[q] = s_acc[ww][q];
      big_acc_signed<L, L>(b, o, 0u);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) part[blockIdx.x * 8 + q] = q < L ? b[q] : 0u;
  }
  if (!arrive_last(a.counter)) return;
  if (threadIdx.x == 0) {
    uint32_t tot[6] = {0u, 0u, 0u, 0u, 0u, 0u};
    for (unsigned int bI = 0; bI < gridDim.x; ++bI) {
      uint32_t o[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) o[q] = q < L ? part[bI * 8 + q] : 0u;
      big_acc_signed<6, 6>(tot, o, 0u);
    }
    // sign-extend a 160-bit residue to 192 bits: the true sum fits W bits
    if (L == 5) tot[5] = (tot[4] & 0x80000000u) ? 0xFFFFFFFFu : 0u;
    int32_t st = PERM_OK;
    const bool aborted = *a.aborted != 0u;
    if (sh.bad_entry) st = PERM_EINVAL;
    else if (aborted) st = stop_status(*a.aborted);
    else if (!sh.zero_row && sh.bound_log2 >= (float)(32 * L - N + 1) - 0.01f) st = PERM_EOVERFLOW;
    uint64_t* out = static_cast<uint64_t*>(a.out);
    if (a.mode == 1) {
      const bool none = sh.bad_entry || aborted;
      out[0] = none ? 0ull : ((uint64_t)tot[1] << 32) | tot[0];
      out[1] = none ? 0ull : ((uint64_t)tot[3] << 32) | tot[2];
      out[2] = none ? 0ull : ((uint64_t)tot[5] << 32) | tot[4];
    } else {
      // sum = (-1)^(n-1) 2^(n-1) perm  (mod 2^W)
      uint32_t v[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) v[q] = tot[q];
      if (((N - 1) & 1) != 0) {
        uint32_t z[6] = {0u, 0u, 0u, 0u, 0u, 0u};
        big_acc_signed<6, 6>(z, v, 0xFFFFFFFFu);
#pragma unroll
        for (int q = 0; q < 6; ++q) v[q] = z[q];
      }
      // v / 2^(n-1): the low n-1 bits are zero by the identity
      const int sh_ = N - 1;
      uint32_t r[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int bit = q * 32 + sh_;
        const int wd = bit >> 5, of = bit & 31;
        uint32_t lo = wd < 6 ? v[wd] : 0u;
        uint32_t hi = wd + 1 < 6 ? v[wd + 1] : 0u;
        r[q] = of ? (lo >> of) | (hi << (32 - of)) : lo;
      }
      // bits above 2^128 of the shifted value must be zero
      uint32_t above = 0u;
      for (int bit = 128 + sh_; bit < 32 * L; ++bit) above |= (v[bit >> 5] >> (bit & 31)) & 1u;
      if (st == PERM_OK && above) st = PERM_EOVERFLOW;
      const bool ok = st == PERM_OK;
      out[0] = ok && !sh.zero_row ? ((uint64_t)r[1] << 32) | r[0] : 0ull;
      out[1] = ok && !sh.zero_row ? ((uint64_t)r[3] << 32) | r[2] : 0ull;
    }
    if (a.status) *a.status = (a.mode == 1 && st == PERM_EOVERFLOW) ? PERM_EOVERFLOW : st;
    *a.counter = 0u;
  }
}

}  // namespace permgpu
