// Sparse real Ryser kernel (Alg. 2, SPARYSER, chunked as Alg. 3 with
// power-of-two chunks, Sec. 3.1.1) on a CCS matrix (Fig. 1).
//
//  * Rows are scaled by a power of two and rounded once to 64-bit fixed point
//    exactly as in the dense kernel, but without the odd-row trick, so a row
//    value is exactly zero when the fixed-point sum is zero.
//  * The row vector lives in shared memory, one int64 per (row, lane) with
//    the lane index fastest (conflict-free), because the rows a column touches
//    are only known at run time.  Each step applies only the nonzeros of the
//    changed column (Alg. 2), from a per-column list staged in shared memory;
//    all lanes of a warp walk the same list (aligned chunks), so the list
//    reads are broadcasts.
//  * Every lane counts its zero rows; while the count is positive the term is
//    exactly zero and the product is skipped.
//  * Quiet rows.  Inside an aligned block of 2^B steps only the columns with
//    Gray bits 0..B-1 change, so B sparse columns (their union of rows small,
//    B in 0..4 from a cost estimate) are moved to those bits (a column
//    permutation leaves the permanent unchanged).  The rows they do not touch stay
//    constant for the whole block: their product is formed once per block and
//    every step multiplies only the touched rows into it (about 2x fewer
//    products at density 0.2).
//  * Products, exact per-step double-double accumulation and the fixed-order
//    reduction are those of the dense real kernel.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "common.cuh"
#include "kernels.h"
#include "real.cuh"

namespace permgpu {

constexpr int kSpBlock = 128;  // threads per CTA (row vector: n x 128 x 8 bytes)
constexpr int kSpWarps = kSpBlock / 32;

struct SpEntry {
  int32_t row;
  int32_t pad;
  long long d;  // +2 Q_ij; the leaving sign is applied by negation
};

struct SpArgs {
  const int32_t* cptrs;
  const int32_t* rids;
  const double* cvals;
  int n;
  int nnz;
  int c;
  int mode;         // 0: write the finished permanent, 1: write the raw range sum (hi, lo)
  int paper_order;  // 1: Alg. 2's own column order (no quiet-row reordering)
  uint64_t g_begin, g_end;  // accumulated steps
  uint64_t k_begin, nchunks;  // visited chunks [k_begin, k_begin + nchunks)
  dd* part;
  unsigned int* counter;
  double* out;
  int32_t* status;
  const volatile uint32_t* abort_word;
  unsigned int* aborted;
  uint64_t budget_ns;
};

struct SpShared {
  int bad;
  int zero_row;
  int sum_s;
  int bound_log2;
};

// Dynamic shared memory: cp[n+1] (int32, column pointers), ent[nnz] (SpEntry),
// base[n] (int64), then the row vectors x[n][kSpBlock] (int64).
__global__ void __launch_bounds__(kSpBlock) ryser_sparse_kernel(SpArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ SpShared sh;
  __shared__ int s_scale[64];
  __shared__ int s_cmap[64];            // Gray bit j -> CCS column
  __shared__ unsigned char s_trow[64];  // rows touched by the columns of bits 0..B-1
  __shared__ unsigned char s_qrow[64];  // the other (quiet) rows
  __shared__ int s_nt, s_nq;
  __shared__ unsigned long long s_tmask;
  const int n = a.n, nnz = a.nnz;
  int32_t* cp = reinterpret_cast<int32_t*>(smem);
  const size_t off_ent = ((sizeof(int32_t) * (n + 1) + 15) / 16) * 16;
  SpEntry* ent = reinterpret_cast<SpEntry*>(smem + off_ent);
  long long* base = reinterpret_cast<long long*>(smem + off_ent + sizeof(SpEntry) * nnz);
  long long* xs = base + n;  // x[i * kSpBlock + tid]

  if (threadIdx.x == 0) {
    sh.bad = 0;
    sh.zero_row = 0;
    sh.sum_s = 0;
    sh.bound_log2 = 0;
  }
  __syncthreads();
  // structure checks (Fig. 1): cptrs[0] = 0, cptrs[n] = nnz, monotone, rows in
  // range and strictly increasing within a column, finite values
  for (int j = threadIdx.x; j <= n; j += kSpBlock) {
    int v = a.cptrs[j];
    cp[j] = v;
    if ((j == 0 && v != 0) || (j == n && v != nnz) || v < 0 || v > nnz) atomicOr(&sh.bad, 1);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += kSpBlock) {
    if (cp[j] > cp[j + 1]) atomicOr(&sh.bad, 1);
  }
  __syncthreads();
  if (!sh.bad) {
    for (int j = threadIdx.x; j < n; j += kSpBlock)
      for (int p = cp[j]; p < cp[j + 1]; ++p) {
        int r = a.rids[p];
        double v = a.cvals[p];
        if (r < 0 || r >= n || (p > cp[j] && r <= a.rids[p - 1]) || !isfinite(v)) atomicOr(&sh.bad, 1);
      }
  }
  __syncthreads();
  // exact column equilibration, full sweeps only (see column_scales): thread j scans column j
  __shared__ int s_cexp[64];
  __shared__ int s_emax, s_csum;
  if (threadIdx.x == 0) {
    s_emax = -100000;
    s_csum = 0;
  }
  __syncthreads();
  int ecol = -100000;
  if (!sh.bad && threadIdx.x < n) {
    double m = 0.0;
    for (int p = cp[threadIdx.x]; p < cp[threadIdx.x + 1]; ++p) m = fmax(m, fabs(a.cvals[p]));
    if (m > 0.0 && isfinite(m)) {
      frexp(m, &ecol);
      atomicMax(&s_emax, ecol);
    }
  }
  __syncthreads();
  if (threadIdx.x < n) {
    const int cj = (a.mode == 0 && ecol > -100000 && s_emax - ecol > kColGap) ? s_emax - ecol : 0;
    s_cexp[threadIdx.x] = cj;
    if (cj) atomicAdd(&s_csum, cj);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    sh.sum_s = s_csum;
    sh.bound_log2 = -s_csum;
  }
  __syncthreads();
  // row scales: thread i scans every column for row i (deterministic sums)
  if (!sh.bad && threadIdx.x < n) {
    const int i = threadIdx.x;
    double absum = 0.0;
    for (int j = 0; j < n; ++j)
      for (int p = cp[j]; p < cp[j + 1]; ++p)
        if (a.rids[p] == i) absum += ldexp(fabs(a.cvals[p]), s_cexp[j]);
    int k = 0;
    if (absum > 0.0) frexp(absum, &k);
    else atomicOr(&sh.zero_row, 1);
    s_scale[i] = 61 - k;
    atomicAdd(&sh.sum_s, 61 - k);
    atomicAdd(&sh.bound_log2, k - 1);
  }
  __syncthreads();
  // column entries (2 Q_ij) and base_i = Q_{i,n-1} - sum_{j<n-1} Q_ij
  if (!sh.bad) {
    for (int j = threadIdx.x; j < n; j += kSpBlock)
      for (int p = cp[j]; p < cp[j + 1]; ++p) {
        int r = a.rids[p];
        long long q = __double2ll_rn(ldexp(a.cvals[p], s_scale[r] + s_cexp[j]));
        ent[p].row = r;
        ent[p].pad = 0;
        ent[p].d = 2 * q;
      }
  }
  __syncthreads();
  if (!sh.bad && threadIdx.x < n) {
    const int i = threadIdx.x;
    long long b = 0;
    for (int j = 0; j < n; ++j)
      for (int p = cp[j]; p < cp[j + 1]; ++p)
        if (ent[p].row == i) b += (j == n - 1) ? ent[p].d / 2 : -(ent[p].d / 2);
    base[i] = b;
  }
  __syncthreads();

  __shared__ int s_B;
  if (threadIdx.x == 0) {
    // Greedily pick up to 4 columns among 0..n-2, each time the one that adds
    // the fewest rows to the touched set; keep the prefix of B columns that
    // minimises the products per step, |T| + (n - |T|) / 2^B + 2.  Those
    // columns take Gray bits 0..B-1 (B <= c); the others keep their order.
    for (int j = 0; j < 64; ++j) s_cmap[j] = j;
    int chosen[4] = {-1, -1, -1, -1};
    unsigned long long masks[5] = {0ull, 0ull, 0ull, 0ull, 0ull};
    const int bmax = (sh.bad || a.paper_order) ? 0 : min(min(a.c, 4), n - 1);
    int B = 0;
    float best_cost = (float)n + 2.0f;
    for (int b = 0; b < bmax; ++b) {
      int best = -1, bestc = 1 << 30;
      for (int j = 0; j < n - 1; ++j) {
        bool used = false;
        for (int q = 0; q < b; ++q) used |= chosen[q] == j;
        if (used) continue;
        unsigned long long m = masks[b];
        for (int p = cp[j]; p < cp[j + 1]; ++p) m |= 1ull << ent[p].row;
        const int cnt = __popcll(m);
        if (cnt < bestc) bestc = cnt, best = j;
      }
      chosen[b] = best;
      masks[b + 1] = masks[b];
      for (int p = cp[best]; p < cp[best + 1]; ++p) masks[b + 1] |= 1ull << ent[p].row;
      const int t_rows = __popcll(masks[b + 1]);
      const float cost = (float)t_rows + (float)(n - t_rows) / (float)(1 << (b + 1)) + 2.0f;
      if (cost < best_cost) best_cost = cost, B = b + 1;
    }
    const unsigned long long tmask = masks[B];
    if (B > 0) {
      int k = 0;
      for (int b = 0; b < B; ++b) s_cmap[k++] = chosen[b];
      for (int j = 0; j < n - 1; ++j) {
        bool used = false;
        for (int q = 0; q < B; ++q) used |= chosen[q] == j;
        if (!used) s_cmap[k++] = j;
      }
      s_cmap[n - 1] = n - 1;
    }
    s_B = B;
    int nt = 0, nq = 0;
    for (int i = 0; i < n; ++i) {
      if ((tmask >> i) & 1ull) s_trow[nt++] = (unsigned char)i;
      else s_qrow[nq++] = (unsigned char)i;
    }
    s_nt = nt;
    s_nq = nq;
    s_tmask = tmask;
  }
  __syncthreads();
  const int nt = s_nt, nq = s_nq;
  const unsigned long long tmask = s_tmask;
  const uint32_t bmask = (1u << s_B) - 1u;

  const bool skip = sh.bad || sh.zero_row || sh.bound_log2 + n > 1000;
  // binary64 exponent of a term: three chains (two over the touched rows, one
  // over the quiet rows) and two merges; see prod_mul for the bookkeeping
  const int F0 = 33 * n + 1022 - 56 - sh.sum_s;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const uint64_t t_start = global_ns();
  const uint64_t warp_id = (uint64_t)(blockIdx.x * kSpBlock + tid) >> 5;
  const uint64_t nwarps = (uint64_t)(gridDim.x * kSpBlock) >> 5;
  const uint64_t ngroups = skip ? 0 : (a.nchunks + 31) / 32;
  const uint32_t nsteps = 1u << a.c;
  dd acc = {0.0, 0.0};

  for (uint64_t q = warp_id; q < ngroups; q += nwarps) {
    if (should_stop(a.abort_word, a.budget_ns, t_start, a.aborted)) break;
    const uint64_t kk = q * 32 + lane;
    const bool active = kk < a.nchunks;
    const uint64_t k = a.k_begin + kk;
    const uint64_t g0 = k << a.c;
    // steps of this chunk inside [g_begin, g_end): local t in [tlo, tlo + tcnt)
    uint32_t tlo, tcnt;
    {
      const uint64_t len = 1ull << a.c;
      const uint64_t lo = a.g_begin > g0 ? a.g_begin - g0 : 0;
      uint64_t hi = a.g_end > g0 ? a.g_end - g0 : 0;
      if (hi > len) hi = len;
      tlo = (uint32_t)lo;
      tcnt = (active && hi > lo) ? (uint32_t)(hi - lo) : 0u;
    }
    const uint32_t kb = (uint32_t)(k & 1u) << a.c;
    const uint32_t gpar = (uint32_t)(g0 & 1u);
    // x at Gray(g0) and its zero count
    for (int i = 0; i < n; ++i) xs[i * kSpBlock + tid] = base[i];
    const uint64_t G = gray64(g0);
    for (int j = (a.c > 0 ? a.c - 1 : 0); j < n - 1; ++j) {
      if ((G >> j) & 1u) {
        const int cj = s_cmap[j];
        for (int p = cp[cj]; p < cp[cj + 1]; ++p) xs[ent[p].row * kSpBlock + tid] += ent[p].d;
      }
    }
    int zeros = 0, zq = 0;  // zero rows in all / in the quiet rows
    for (int i = 0; i < n; ++i) {
      const int z = xs[i * kSpBlock + tid] == 0;
      zeros += z;
      zq += ((tmask >> i) & 1ull) ? 0 : z;
    }

    Prod pq;  // product of the quiet rows of the current block
    uint32_t negq = 0, eposq = 0;
    prod_init(pq);
    for (uint32_t t = 0; t < nsteps; ++t) {
      if (t) {
        const int j = s_cmap[__ffs(t) - 1];
        const bool leave = ((t | kb) >> __ffs(t)) & 1u;  // bit j + 1 of g
        for (int p = cp[j]; p < cp[j + 1]; ++p) {  // Alg. 2: nonzeros of column j only
          const SpEntry e = ent[p];
          long long* xp = xs + e.row * kSpBlock + tid;
          const long long old = *xp;
          const long long nv = leave ? old - e.d : old + e.d;
          *xp = nv;
          const int dz = (nv == 0) - (old == 0);
          zeros += dz;
          zq += ((tmask >> e.row) & 1ull) ? 0 : dz;
        }
      }
      if ((t & bmask) == 0u) {
        // a new block: the quiet rows are constant until its end
        prod_init(pq);
        negq = 0;
        eposq = 0;
        // (skipped while a quiet row is zero: then every term of the block is)
        for (int k = 0; k < (zq == 0 ? nq : 0); ++k) {
          const long long ya = xs[s_qrow[k] * kSpBlock + tid];
          const uint32_t ma = (uint32_t)(ya >> 63);
          const unsigned long long aa = (unsigned long long)((ya ^ (long long)(int32_t)ma) - (long long)(int32_t)ma);
          negq += ma;
          eposq += prod_mul(pq, (uint32_t)aa, (uint32_t)(aa >> 32));
        }
      }
      if (zeros == 0 && t - tlo < tcnt) {
        Prod pa, pb;
        prod_init(pa);
        prod_init(pb);
        uint32_t neg = negq, epos = eposq;
        int k = 0;
        for (; k + 1 < nt; k += 2) {
          const long long ya = xs[s_trow[k] * kSpBlock + tid], yb = xs[s_trow[k + 1] * kSpBlock + tid];
          const uint32_t ma = (uint32_t)(ya >> 63), mb = (uint32_t)(yb >> 63);
          const unsigned long long aa = (unsigned long long)((ya ^ (long long)(int32_t)ma) - (long long)(int32_t)ma);
          const unsigned long long ab = (unsigned long long)((yb ^ (long long)(int32_t)mb) - (long long)(int32_t)mb);
          neg = neg + ma + mb;
          epos += prod_mul(pa, (uint32_t)aa, (uint32_t)(aa >> 32));
          epos += prod_mul(pb, (uint32_t)ab, (uint32_t)(ab >> 32));
        }
        if (k < nt) {
          const long long ya = xs[s_trow[k] * kSpBlock + tid];
          const uint32_t ma = (uint32_t)(ya >> 63);
          const unsigned long long aa = (unsigned long long)((ya ^ (long long)(int32_t)ma) - (long long)(int32_t)ma);
          neg += ma;
          epos += prod_mul(pa, (uint32_t)aa, (uint32_t)(aa >> 32));
        }
        epos += prod_mul(pa, pb.m0, pb.m1);
        epos += prod_mul(pa, pq.m0, pq.m1);
        const int f = F0 + (int)epos;
        const uint32_t signbit = (neg ^ t ^ gpar) << 31;
        double th, tl;
        prod_to_dd(pa, (uint32_t)max(f, 0), signbit, th, tl);
        dd_acc(acc, th, tl);
      }
    }
    acc = dd_make(acc.hi, acc.lo);
  }

  // reduction (fixed order): warps -> CTA -> last CTA
  __shared__ dd s_w[kSpWarps];
  dd v = dd_warp_sum(acc);
  if (lane == 0) s_w[tid >> 5] = v;
  __syncthreads();
  if (tid == 0) {
    dd b = {0.0, 0.0};
    for (int w = 0; w < kSpWarps; ++w) b = dd_add(b, s_w[w]);
    a.part[blockIdx.x] = b;
  }
  if (!arrive_last(a.counter)) return;
  if (tid < 32) {
    dd tot = dd_sum_partials(a.part, gridDim.x);
    if (tid == 0) {
      int32_t st = PERM_OK;
      if (sh.bad) st = PERM_EINVAL;
      else if (!sh.zero_row && sh.bound_log2 + n > 1000) st = PERM_ERANGE;
      else if (*a.aborted) st = stop_status(*a.aborted);
      const double f = (n & 1) ? 2.0 : -2.0;
      if (a.mode == 0) {
        a.out[0] = st != PERM_OK ? __longlong_as_double(0x7ff8000000000000ll)
                   : (sh.zero_row ? 0.0 : (tot.hi + tot.lo) * f);
      } else {
        a.out[0] = st != PERM_OK ? __longlong_as_double(0x7ff8000000000000ll) : (sh.zero_row ? 0.0 : tot.hi);
        a.out[1] = (st != PERM_OK || sh.zero_row) ? 0.0 : tot.lo;
      }
      if (a.status) *a.status = st;
      *a.counter = 0u;
    }
  }
}

__global__ void sparse_trivial_kernel(int mode, double* out, int32_t* status) {
  if (threadIdx.x == 0) {
    if (mode == 0) out[0] = 1.0;
    else out[0] = out[1] = 0.0;
    if (status) *status = PERM_OK;
  }
}

// One sparse launch over the steps [g0, g1) (mode 0: the permanent, 1: the
// raw range sum).
static int sparse_launch(int n, const int32_t* cptrs, const int32_t* rids, const double* cvals, int64_t nnz,
                         uint64_t g0, uint64_t g1, int mode, int paper_order, double* out, int32_t* status,
                         cudaStream_t s) {
  const size_t off_ent = ((sizeof(int32_t) * (n + 1) + 15) / 16) * 16;
  const size_t smem = off_ent + sizeof(SpEntry) * (size_t)nnz + sizeof(long long) * n +
                      sizeof(long long) * (size_t)n * kSpBlock;
  static std::mutex mu;
  int nb = 0, dev = 0, sms = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (cudaFuncSetAttribute(ryser_sparse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
      cudaGetLastError();
      return PERM_ERANGE;  // does not fit shared memory
    }
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ryser_sparse_kernel, kSpBlock, smem) != cudaSuccess ||
        nb <= 0)
      return PERM_ECUDA;
  }
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PERM_ECUDA;
  const int grid_full = sms * nb;
  const int c = plan_chunk_exponent(n, g1 - g0, grid_full * kSpWarps);
  const uint64_t k_begin = g0 >> c;
  const uint64_t k_end = (g1 + (1ull << c) - 1) >> c;
  const uint64_t nchunks = g1 > g0 ? k_end - k_begin : 0;
  const uint64_t need = ((nchunks + 31) / 32 + kSpWarps - 1) / kSpWarps;
  const int grid = (int)(need < (uint64_t)grid_full ? (need > 0 ? need : 1) : grid_full);
  void* ws = nullptr;
  const size_t bytes = sizeof(dd) * (size_t)grid + 16;
  if (cudaMallocAsync(&ws, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return PERM_ENOMEM;
  }
  unsigned int* counter = reinterpret_cast<unsigned int*>(static_cast<char*>(ws) + sizeof(dd) * (size_t)grid);
  if (cudaMemsetAsync(counter, 0, 2 * sizeof(unsigned int), s) != cudaSuccess) {
    cudaFreeAsync(ws, s);
    return PERM_ECUDA;
  }
  SpArgs args;
  memset(&args, 0, sizeof(args));
  args.cptrs = cptrs;
  args.rids = rids;
  args.cvals = cvals;
  args.n = n;
  args.nnz = (int)nnz;
  args.c = c;
  args.mode = mode;
  args.paper_order = paper_order;
  args.g_begin = g0;
  args.g_end = g1;
  args.k_begin = k_begin;
  args.nchunks = nchunks;
  args.part = static_cast<dd*>(ws);
  args.counter = counter;
  args.out = out;
  args.status = status;
  args.abort_word = current_abort_word();
  args.aborted = counter + 1;
  args.budget_ns = current_time_budget();
  void* params[] = {&args};
  cudaError_t e = cudaLaunchKernel(reinterpret_cast<const void*>(ryser_sparse_kernel), dim3(grid), dim3(kSpBlock),
                                   params, smem, s);
  cudaError_t f = cudaFreeAsync(ws, s);
  if (e != cudaSuccess || f != cudaSuccess) {
    cudaGetLastError();
    return PERM_ECUDA;
  }
  return PERM_OK;
}

static int sparse_check(int n, const int32_t* cptrs, const int32_t* rids, const double* cvals, int64_t nnz,
                        const double* out) {
  if (n < 0 || n > PERM_NMAX) return PERM_ERANGE;
  if (!out || (n > 0 && !cptrs) || nnz < 0 || nnz > (int64_t)n * n || (nnz > 0 && (!rids || !cvals)))
    return PERM_EINVAL;
  return PERM_OK;
}

}  // namespace permgpu

using namespace permgpu;

extern "C" int perm_sparse(int n, const int32_t* cptrs, const int32_t* rids, const double* cvals, int64_t nnz,
                           double* out, int32_t* status, void* stream) {
  int rc = sparse_check(n, cptrs, rids, cvals, nnz, out);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n == 0) {
    sparse_trivial_kernel<<<1, 32, 0, s>>>(0, out, status);
    return cudaGetLastError() == cudaSuccess ? PERM_OK : PERM_ECUDA;
  }
  return sparse_launch(n, cptrs, rids, cvals, nnz, 0, 1ull << (n - 1), 0, 0, out, status, s);
}

extern "C" int perm_sparse_range(int n, const int32_t* cptrs, const int32_t* rids, const double* cvals, int64_t nnz,
                                 uint64_t g_begin, uint64_t g_end, int flags, double* partial, int32_t* status,
                                 void* stream) {
  int rc = sparse_check(n, cptrs, rids, cvals, nnz, partial);
  if (rc) return rc;
  if (flags & ~PERM_SPARSE_PAPER_ORDER) return PERM_EINVAL;
  const uint64_t N = n > 0 ? 1ull << (n - 1) : 0;
  if (g_begin > g_end || g_end > N) return PERM_ERANGE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n == 0 || g_begin == g_end) {
    sparse_trivial_kernel<<<1, 32, 0, s>>>(1, partial, status);
    return cudaGetLastError() == cudaSuccess ? PERM_OK : PERM_ECUDA;
  }
  return sparse_launch(n, cptrs, rids, cvals, nnz, g_begin, g_end, 1, (flags & PERM_SPARSE_PAPER_ORDER) ? 1 : 0,
                       partial, status, s);
}
