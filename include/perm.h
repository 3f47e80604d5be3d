/*
 * perm.h - C ABI of the GB300 permanent library (libperm.so).
 *
 * The library evaluates the permanent of an n x n matrix,
 *
 *     perm(A) = sum over permutations sigma of prod_i a_{i,sigma(i)}      (Eq. 1)
 *
 * with Ryser's inclusion-exclusion formula (Eq. 2) in the Nijenhuis-Wilf form
 * (Eq. nwx): a row vector x, started at x_i = a_{i,n} - r_i/2, is updated by
 * one column per step while the 2^(n-1) column subsets of columns 1..n-1 are
 * visited in binary-reflected Gray-code order, Gray_g = g xor (g >> 1)
 * (Sec. 2, Table 1, Alg. 1); every step adds (-1)^g prod_i x_i to a sum and
 * perm(A) = 2 (-1)^(n-1) times the sum.  The 2^(n-1) steps are split into
 * aligned chunks of 2^c steps (Alg. 3, with the power-of-two chunks of
 * Sec. 3.1.1), each started from the x of its first Gray code, and the chunk
 * sums are reduced on the device.
 *
 * Conventions for every entry point:
 *   - Matrices are row-major, a_{i,j} at A[i*n + j], 0-based; the paper's
 *     column n is column n-1 here.
 *   - "device" pointers are CUDA device (or managed) memory on the current
 *     device; "host" pointers are ordinary host memory.  The caller owns every
 *     buffer and the library never frees one.  Only a batched plan (its bound
 *     input / output buffers) and the registered abort word keep a caller
 *     pointer beyond the call, as documented at those entry points.
 *   - stream is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Device-pointer calls are stream-ordered and return without waiting for
 *     the GPU; they take their scratch memory with cudaMallocAsync on that
 *     stream and release it with cudaFreeAsync on the same stream.
 *   - The return value is a perm_status_t for errors found on the host
 *     (argument checks, CUDA launch errors).  Errors that depend on the matrix
 *     values are found on the GPU and written to *status (device int32,
 *     optional: pass NULL to skip it) when the call completes on the stream.
 *   - n ranges over 0..63 (n_max = 63 as in Sec. 3.2); perm of the 0 x 0
 *     matrix is 1.
 *   - No call traps, aborts or prints; nothing is thrown across the ABI.
 */
#ifndef PERM_H
#define PERM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PERM_ABI_VERSION 4
#define PERM_NMAX 63

typedef enum {
  PERM_F64 = 0,  /* real binary64 entries                                   */
  PERM_C128 = 1, /* complex entries, (re, im) binary64 pairs                 */
  PERM_BIN = 2,  /* 0/1 entries as uint8; the result is exact               */
  PERM_F64X = 3  /* real binary64 entries, extended-precision products and a
                    double-double result (Sec. 5's quad inner product)       */
} perm_type_t;

typedef enum {
  PERM_OK = 0,
  PERM_EINVAL = 1,    /* bad argument; non-finite entry; a BIN entry not 0/1 */
  PERM_ERANGE = 2,    /* n out of 0..63, range out of [0, 2^(n-1)), or a
                         binary64 result that can overflow                      */
  PERM_EOVERFLOW = 3, /* BIN: the permanent may not fit 128 bits              */
  PERM_ECUDA = 4,     /* a CUDA call failed                                    */
  PERM_ENOMEM = 5,    /* scratch allocation failed                             */
  PERM_EABORTED = 6,  /* stopped early by the word of perm_set_abort_word      */
  PERM_ETIMEOUT = 7   /* stopped when the budget of perm_set_time_budget ran out */
} perm_status_t;

/*
 * perm - permanent of one dense n x n matrix (Eq. 1 by Alg. 1 + Alg. 3).
 *
 *   A      device; PERM_F64, PERM_F64X: double[n*n]; PERM_C128: double[2*n*n]
 *          as (re, im) pairs; PERM_BIN: uint8_t[n*n] holding only 0 and 1.
 *   out    device; PERM_F64: double[1]; PERM_C128: double[2] = (re, im);
 *          PERM_BIN: uint64_t[2] = the permanent as a little-endian unsigned
 *          128-bit integer; PERM_F64X: double[2] = (hi, lo), the permanent as
 *          the unevaluated sum hi + lo with |lo| <= ulp(hi) / 2.
 *   status device int32_t[1] or NULL; receives PERM_OK, PERM_EINVAL (a
 *          non-finite entry, or a BIN entry other than 0/1: out is then NaN /
 *          zero), PERM_ERANGE (PERM_F64/F64X/C128: the largest possible term
 *          exceeds the binary64 range; out is then NaN) or PERM_EOVERFLOW
 *          (PERM_BIN only: perm(A) may be >= 2^128; out is then zero).
 *
 * Real and complex entries are converted once to 64-bit fixed point with a
 * power-of-two scale per row (error at most 2^-60 of the row's absolute sum)
 * and the row vector x is kept exactly; columns whose largest entry lies more
 * than a factor 2 below the largest column's are first scaled by an exact
 * power of two up to its level (perm(A D) = perm(A) det D for a diagonal D of
 * powers of two, taken back out of the result exactly), which keeps their
 * bits and avoids the cancellation a dominant column causes; products carry 62-bit mantissas and
 * the signed sum is accumulated in binary64 with a double-double carry.
 * PERM_F64X uses the same fixed-point rows (column n-1 rounded to nearest,
 * so a row is exact when every a_ij 2^(60-k) is an integer, k the binary
 * exponent of the row's absolute sum) with 128-bit product mantissas
 * (2^-123 per factor), splits every term into a double-double without
 * losing more than 2^-105 of it, and renormalises the double-double after
 * every step; it costs about 2.1x PERM_F64.
 * Binary matrices run in exact wrap-around integer arithmetic (192 bits).
 * Results are bitwise reproducible for a given n, type and GPU model.
 */
int perm(const void* A, int n, int type, void* out, int32_t* status, void* stream);

/*
 * perm_range - unscaled partial sum of the steps g in [g_begin, g_end)
 * (0 <= g_begin <= g_end <= 2^(n-1)), so that ranges can be spread over GPUs,
 * processes or time (Secs. 3.3 and 6.3: the iteration space is split first per GPU;
 * the only exchange is the final sum).
 *
 *   partial device;
 *     PERM_F64, PERM_F64X: double[2] = (hi, lo) of  sum_g (-1)^g prod_i x_i(g);
 *     PERM_C128: double[4]   = (re hi, re lo, im hi, im lo) of the same sum;
 *     PERM_BIN:  uint64_t[3] = sum_g (-1)^g prod_i x'_i(g) modulo 2^192,
 *                little-endian, with the doubled integer rows x' = 2x.
 *   x_i(g) is Alg. 1's row vector after the subsets up to Gray_g, with
 *   x_i(0) = a_{i,n-1} - (sum_j a_{i,j}) / 2.  The matrix is staged without
 *   perm()'s column equilibration, which changes individual terms: the
 *   partials are sums of these very terms (only perm() of the whole sweep
 *   balances the columns).
 *   status as for perm(); for PERM_BIN it reports PERM_EOVERFLOW when the
 *   combined sum may not determine perm(A) (the partial itself stays exact).
 */
int perm_range(const void* A, int n, int type, uint64_t g_begin, uint64_t g_end, void* partial,
               int32_t* status, void* stream);

/*
 * perm_combine - host-side reduction of perm_range partials that together
 * cover [0, 2^(n-1)) exactly once, in the order given, into the perm() output
 * format: multiply by 2 (-1)^(n-1) (Alg. 1) for real and complex (PERM_F64X:
 * the double-double sum, scaled exactly, as (hi, lo)); for BIN add
 * modulo 2^192, check that the low n-1 bits are zero (PERM_EINVAL otherwise),
 * shift them out, apply (-1)^(n-1) and check the value fits 128 bits
 * (PERM_EOVERFLOW otherwise).
 *
 *   partials host, count consecutive partials of the perm_range layout.
 *   out      host, the perm() layout.
 */
int perm_combine(int type, int n, const void* partials, int count, void* out);

/*
 * perm_sparse - permanent of an n x n real matrix given in compressed column
 * storage (Fig. 1): column j holds rows rids[cptrs[j] .. cptrs[j+1]-1]
 * (strictly increasing) with values cvals[...]; cptrs[0] = 0, cptrs[n] = nnz.
 * Alg. 2: each step updates only the nonzeros of the changed column, and the
 * product is skipped while some x_i is exactly zero (such a term is zero).
 *
 *   cptrs, rids, cvals  device; int32_t[n+1], int32_t[nnz], double[nnz].
 *   out                 device double[1];  status as for perm().
 * The CCS structure is checked on the device: a malformed one gives
 * PERM_EINVAL in *status and NaN in out.
 */
int perm_sparse(int n, const int32_t* cptrs, const int32_t* rids, const double* cvals, int64_t nnz,
                double* out, int32_t* status, void* stream);

/*
 * perm_sparse_range - the unscaled partial sum of the sparse sweep over the
 * steps g in [g_begin, g_end) (0 <= g_begin <= g_end <= 2^(n-1)), written to
 * partial (device double[2] = (hi, lo)), for splitting one sparse permanent
 * over GPUs, processes or time like perm_range (Secs. 3.3 and 6.3).
 *   flags 0: the kernel's own column order.  Up to four sparse columns
 *       (chosen from the matrix alone, deterministically) take Gray bits
 *       0..B-1 so that the rows they do not touch stay constant for 2^B steps
 *       (a column permutation leaves the permanent unchanged); the remaining
 *       columns follow in their order.  Partials of any partition of
 *       [0, 2^(n-1)) made with flags 0 combine to perm(A), as perm_sparse.
 *   flags PERM_SPARSE_PAPER_ORDER: Alg. 2's own order, Gray bit j <-> column j
 *       (the steps of perm_range on the dense form); slower at low density.
 * Like perm_range, ranges are staged without perm_sparse's column
 * equilibration.  Partials combine with perm_combine(PERM_F64, ...).  status
 * as perm_sparse;
 * PERM_EINVAL for unknown flags, PERM_ERANGE for a bad range.
 */
#define PERM_SPARSE_PAPER_ORDER 1
int perm_sparse_range(int n, const int32_t* cptrs, const int32_t* rids, const double* cvals, int64_t nnz,
                      uint64_t g_begin, uint64_t g_end, int flags, double* partial, int32_t* status,
                      void* stream);

/*
 * Batched permanents (boson-sampling style: thousands of small k x k
 * matrices of uneven sizes; complex, or real).  Each matrix is the sweep of perm() (Alg. 1 over
 * complex entries, Alg. 3 chunks of Sec. 3.1.1); all of them run in one
 * CUDA-graph replay: a prep kernel (fixed-point tables), one persistent
 * kernel that pops work items (32 matrices of one size per warp for short
 * sweeps, 32 aligned Gray chunks of one matrix per warp for long ones,
 * longest first) from an atomic counter, and a finish kernel that adds each
 * matrix's item partials in a fixed order.  The prep kernel equilibrates the
 * lines a unit's sweep toggles as perm() does (columns; for the repeated-row
 * sweeps of a labelled plan, the rows, equal rows alike) and takes the scale
 * back out of the result exactly.
 *
 * perm_batched_plan_create - build a plan (host call; allocates the plan's
 *   device buffers and captures the graph; synchronous).
 *     type       PERM_C128 or PERM_F64 (one type per plan).
 *     ns_host    host int[count], sizes k in 1..32.
 *     A_packed   device; PERM_C128: double pairs, PERM_F64: doubles; matrix
 *                m is row-major and starts at element offsets_host[m]
 *                (host int64[count]).
 *     out        device; PERM_C128: double[2*count], (re, im) of perm of
 *                every matrix; PERM_F64: double[count].
 *     status     device int32[count] or NULL (perm() status per matrix).
 *   A_packed, out and status are the plan's default buffers: a
 *   perm_batched() call that passes NULL for one of them uses the default.
 * perm_batched_plan_create_labeled - the same, with row_labels_host (host
 *   int32[sum of ns], the rows of matrix 0, then matrix 1, ...): rows of one
 *   matrix with equal labels must be equal (checked on the device: PERM_EINVAL
 *   in its status otherwise).  A matrix whose distinct rows occur mu_r times
 *   is then summed over the multiplicities (Glynn's form of Eq. 2 grouped by
 *   the number of copies of each row with sign -1, weights C(mu_r, k_r)),
 *   1/2 prod_r (mu_r + 1) terms instead of 2^(k-1) (at most 64 sweeps per
 *   matrix, each of at least 2^min(k-1, 8) steps: further repeated rows are
 *   swept as ordinary Gray bits, and a matrix where this does not pay keeps
 *   the plain sweep, its labels still checked); results agree with the
 *   unlabelled plan to the accuracy of the kernels, not bitwise.
 *   row_labels_host NULL: PERM_EINVAL.
 * perm_batched_units - host only (no device call): the sweep units that a
 *   labelled plan builds for one k x k matrix with row labels `labels`
 *   (host int32[k], or NULL for all rows distinct).  Returns the number of
 *   units (only the first max_units are written) or -status.  For unit u:
 *   gray_bits[u] (its sweep has 2^gray_bits steps), weight[u] (its partial
 *   sum is multiplied by weight[u] before the factor 2 (-1)^(k-1)), and
 *   desc_off[u]: -1 for the plain sweep of A, else the offset in desc
 *   (host int32[desc_cap]) of f, G, t_0..t_{G-1}, R, (r, c) x R: the sweep of
 *   the transposed matrix with base row f, toggled rows t_j, and rows r added
 *   c times to every column sum (x_j = (a_fj + sum_r c a_rj + sum_t d_t a_tj) / 2,
 *   d_t = -1 at step 0).  -PERM_ENOMEM if desc_cap is too small.
 * perm_batched - replay the plan's graph on stream (allocates nothing).
 *   A_packed, out, status: device buffers of this call, laid out as at plan
 *   creation (the same sizes, the same element offsets of every matrix); NULL
 *   selects the plan's default buffer.  When they (or the registered abort
 *   word or time budget) differ from the previous replay's, the kernel nodes
 *   of the instantiated graph are updated in place before the launch
 *   (cudaGraphExecKernelNodeSetParams): no capture, no allocation, no wait.
 *   Replays of one plan must be ordered (they share the plan's work queue and
 *   partial sums).  A stopped replay (abort word, time budget) reports
 *   PERM_EABORTED / PERM_ETIMEOUT for every matrix, out NaN.
 * perm_batched_autotune - time the candidate chunk exponents and the
 *   one-matrix-per-lane mode of every size class on the plan's own matrices
 *   (rounds timed runs each), keep the fastest, rebuild the queue and
 *   recapture.  Overwrites out.  Synchronous.
 * perm_batched_plan_info - the choice for size k: *mode (1 = one matrix per
 *   lane, 0 = chunked), *c (chunk exponent), *nitems (queue length).
 * perm_batched_plan_destroy - free the plan (NULL is ignored).
 */
typedef struct perm_batch_plan perm_batch_plan;
int perm_batched_plan_create(perm_batch_plan** plan, int type, const int* ns_host, int count, const void* A_packed,
                             const int64_t* offsets_host, void* out, int32_t* status);
int perm_batched_plan_create_labeled(perm_batch_plan** plan, int type, const int* ns_host, int count,
                                     const void* A_packed, const int64_t* offsets_host, void* out, int32_t* status,
                                     const int32_t* row_labels_host);
int perm_batched_units(int k, const int32_t* labels, int max_units, int32_t* gray_bits, double* weight,
                       int32_t* desc, int desc_cap, int32_t* desc_off);
int perm_batched(perm_batch_plan* plan, const void* A_packed, void* out, int32_t* status, void* stream);
int perm_batched_autotune(perm_batch_plan* plan, int rounds, void* stream);
int perm_batched_plan_info(const perm_batch_plan* plan, int k, int* mode, int* c, int* nitems);
void perm_batched_plan_destroy(perm_batch_plan* plan);

/*
 * perm_grad - perm(A) and its full gradient G = d perm(A) / dA in one
 * Gray-code sweep: G_kl = perm of A without row k and column l.
 * Differentiating Eq. nwx (x_i = (1/2) sum_l delta_l a_il) gives
 *   G_kl = (-1)^(n-1) sum_g (-1)^g delta_l(g) prod_{i != k} x_i(g),
 * accumulated with per-chunk running prefixes so each step costs O(n)
 * additions.  The paper has no gradient; the sweep and its chunking are those
 * of Alg. 1 / Alg. 3.  The permanent is returned through the row expansion
 * perm = sum_l a_0l G_0l (its error follows G's, not perm()'s).  Columns are
 * equilibrated as in perm(); since every minor of A D is det D / d_l times
 * that of A, G is scaled back column by column, exactly.
 *   type    PERM_F64 or PERM_C128 (interleaved re, im); 0 <= n <= 32.
 *   A       device, n*n elements row-major;  out device, one element;
 *   G       device, n*n elements row-major (the holomorphic derivative for
 *           complex A: the gradient of a real loss L is conj(G) dL/dperm);
 *   status  optional device int32: PERM_EINVAL for a non-finite entry (out and
 *           G then NaN), PERM_ERANGE when the result would leave binary64.
 * Allocates a workspace with cudaMallocAsync on `stream`; stream-ordered.
 * Returns PERM_EINVAL / PERM_ERANGE for bad arguments before any launch.
 */
int perm_grad(const void* A, int n, int type, void* out, void* G, int32_t* status, void* stream);

/*
 * perm_grad_batched - perm_grad of `count` matrices of one order n, packed
 * back to back (matrix p at A + p*n*n elements; out[p]; G at G + p*n*n).
 * One sweep launch covers the whole batch (chunks of every matrix share the
 * grid), then one finishing launch; status is the worst over the batch.
 */
int perm_grad_batched(const void* A, int n, int count, int type, void* out, void* G, int32_t* status,
                      void* stream);

/*
 * perm_grad_batched_mixed - perm_grad of `count` matrices of mixed orders.
 *   ns_host       host int[count], orders 0..32;
 *   A_packed      device; matrix m (row-major) starts at element
 *                 offsets_host[m] (host int64[count]);
 *   G_packed      device; gradient m is written at the same element offset;
 *   out           device, count elements (perm of each matrix);
 *   status        optional device int32: the first failing order's code.
 * The host groups the matrices by order; each group is gathered into a
 * contiguous batch, swept by one perm_grad_batched launch and scattered
 * back.  A one-shot gradient plan (below): allocates its buffers and waits
 * for the stream before returning; use a plan to avoid both.
 */
int perm_grad_batched_mixed(int type, const int* ns_host, int count, const void* A_packed,
                            const int64_t* offsets_host, void* out, void* G_packed, int32_t* status,
                            void* stream);

/*
 * Gradient plans: perm_grad_batched_mixed without allocation or waiting per
 * call, for training loops that evaluate the same shapes many times.
 * perm_grad_plan_create - (host call, synchronous) group `count` matrices of
 *   orders ns_host[m] (0..32) at element offsets offsets_host[m] (the layout of
 *   perm_grad_batched_mixed), choose each group's launch shape and allocate
 *   every device buffer the runs need (gather / scatter buffers, index arrays,
 *   one sweep workspace shared by the groups).
 * perm_grad_plan_run - for caller buffers A_packed, G_packed (same offsets)
 *   and out (count elements): per order, gather, one fused sweep
 *   (perm_grad_batched's kernels), scatter; then the status (the first
 *   failing order's code).  Stream-ordered: no allocation, no wait.  Runs of
 *   one plan must be ordered (they share its buffers).
 * perm_grad_plan_destroy - free the plan (NULL is ignored); call it after the
 *   plan's last run has completed.
 */
typedef struct perm_grad_plan perm_grad_plan;
int perm_grad_plan_create(perm_grad_plan** plan, int type, const int* ns_host, int count,
                          const int64_t* offsets_host);
int perm_grad_plan_run(perm_grad_plan* plan, const void* A_packed, void* out, void* G_packed, int32_t* status,
                       void* stream);
void perm_grad_plan_destroy(perm_grad_plan* plan);

/*
 * Sparse preprocessing (Sec. 4; host-side graph work, leaves on the GPU).
 *
 * perm_decomp_create builds, from a HOST CCS matrix (same validation as
 * perm_sparse; entries must be finite), the decomposition of Sec. 4:
 *  - Dulmage-Mendelsohn (Sec. 4.1): entries that lie on no perfect matching
 *    are removed; the rest is block-diagonal up to permutation, one block per
 *    strongly connected component of the matched row/column graph, and
 *    perm(A) = prod over blocks of perm(block).  No perfect matching:
 *    structurally_zero = 1 and perm = 0.
 *  - Forbert-Marx (Sec. 4.2, Eq. expand, Alg. 4): inside a block, rows or
 *    columns with at most four nonzeros are expanded away; every block becomes
 *    a sum of coefficient * perm(leaf).  At most max_leaves leaves are made
 *    (<= 0: 4096); past that, the current matrix is kept as a leaf
 *    (truncated = 1).
 * perm_decomp_eval computes every leaf of order >= 2 on the GPU (dense kernel
 * at density >= 30 %, sparse kernel otherwise) on `stream`, waits for them,
 * and writes perm(A) to the HOST double *out.  Blocking.
 * perm_sparse_decomp = create + eval + destroy (info optional).
 * Ownership: the handle owns its matrices; leaf / filtered copy out to
 * caller-owned host buffers (n*n doubles).
 */
typedef struct perm_decomp perm_decomp;
typedef struct {
  int n, nblocks, nleaves, max_leaf_n, structurally_zero, truncated;
  int64_t removed_nnz;  /* entries removed by the Dulmage-Mendelsohn step */
  double leaf_steps;    /* sum over leaves of order k >= 1 of 2^(k-1) */
  double plain_steps;   /* 2^(n-1): the sweep without preprocessing */
} perm_decomp_info_t;
int perm_decomp_create(perm_decomp** d, int n, const int32_t* cptrs, const int32_t* rids, const double* cvals,
                       int64_t nnz, int max_leaves);
int perm_decomp_info(const perm_decomp* d, perm_decomp_info_t* info);
int perm_decomp_leaf(const perm_decomp* d, int index, int* n, int* block, double* coef, double* A);
int perm_decomp_filtered(const perm_decomp* d, double* A);
int perm_decomp_eval(perm_decomp* d, double* out, void* stream);
void perm_decomp_destroy(perm_decomp* d);
int perm_sparse_decomp(int n, const int32_t* cptrs, const int32_t* rids, const double* cvals, int64_t nnz,
                       double* out, perm_decomp_info_t* info, void* stream);

/*
 * perm_host - perm() on host buffers: copies A in, runs perm() on stream,
 * copies the result out and waits.  Returns the device status as well.
 *   A_host   host, layout as perm()'s A;  out_host  host, layout as perm()'s out.
 */
int perm_host(const void* A_host, int n, int type, void* out_host, void* stream);

/*
 * perm_f64_noalloc - perm(A, n, PERM_F64, out, status, stream) without any
 * allocation.  The paper has no counterpart: this entry point exists for
 * callers that may not call the CUDA allocator, e.g. code running under a
 * framework that has reserved all device memory for its own pool, or loops
 * that forbid allocation once they have started.  Arguments, results and
 * *status are those of perm() for real matrices.
 *
 * Its scratch is a fixed 64 KiB array in the library's device memory (room
 * for 4096 CTA partials); a launch that would need more returns PERM_ENOMEM
 * before doing anything.  The array is shared by every call on a device and
 * keeps the last call's contents: calls whose work overlaps on the GPU
 * (other streams, unordered host threads) race on it and must be ordered by
 * the caller.  The first call on each device looks the array up with
 * cudaGetSymbolAddress; make that first call before any stream capture.
 */
int perm_f64_noalloc(const double* A, int n, double* out, int32_t* status, void* stream);

/*
 * perm_pipe_peaks - measured throughput of the pipes the kernels use, the
 * denominators of the benchmark's roofline fractions (measurement
 * infrastructure; the paper has no counterpart).  Runs microbenchmarks on the
 * current device (8 independent chains of one instruction per thread, 4 CTAs
 * of 256 threads per SM, best of 3) and writes lane-instructions per second:
 *   out[0] fma.rn.f64, out[1] add.rn.f64, out[2] mad.lo.u32,
 *   out[3] mad.wide.u32, out[4] shf.l.wrap.b32  (first count entries).
 *   out  host double[count], 1 <= count <= 5; an entry that could not be
 *        timed (a CUDA error) is NaN.  Waits for the stream.
 */
int perm_pipe_peaks(double* out, int count, void* stream);

/*
 * Cancellation (no counterpart in the paper; a service around Alg. 3's chunk
 * loop).  perm_set_abort_word registers a word of page-locked MAPPED host
 * memory (cudaHostAlloc with cudaHostAllocMapped, or perm_abort_word_alloc);
 * NULL unregisters it.  The sweeps of perm, perm_range, perm_sparse,
 * perm_sparse_range and perm_f64_noalloc launched afterwards read it once per
 * chunk group and warp, the batched replays once per work item and warp, the
 * gradient sweeps once per block-item and CTA; when it is nonzero they stop
 * and report PERM_EABORTED (out NaN, or zero for 0/1; a batched replay marks
 * every matrix of the plan).  Setting the word to nonzero from the host while
 * a launch runs ends that launch early.  Nothing waits on the word.  Returns
 * PERM_EINVAL when the pointer is not mapped host memory.  One word for the
 * process, read at every launch (a batched plan reads it at every
 * perm_batched call).
 * perm_abort_word_alloc / perm_abort_word_free - allocate (zeroed) / free
 * such a word (freeing the registered word unregisters it).
 */
int perm_set_abort_word(volatile uint32_t* host_mapped);

/*
 * perm_set_time_budget - a time budget for every sweep launched afterwards
 * (the paper's largest run took 1.63 days, Secs. 1 and 6.3; a service needs a
 * bound).  Each warp reads the GPU's nanosecond timer between its chunk groups
 * (Alg. 3's chunk loop) and stops once more than `nanoseconds` have passed
 * since it started; the launch then reports PERM_ETIMEOUT (out NaN, or zero
 * for 0/1), its partial results discarded.  Work already done in a group
 * finishes, so a launch overruns its budget by at most one chunk group.
 * 0 (the default) means no budget.  One budget for the process; it applies to
 * perm, perm_range, perm_sparse, perm_sparse_range, perm_f64_noalloc, the
 * batched replays and the gradient sweeps, like the abort word.  Returns
 * PERM_OK.
 */
int perm_set_time_budget(uint64_t nanoseconds);
int perm_abort_word_alloc(volatile uint32_t** host_word);
int perm_abort_word_free(volatile uint32_t* host_word);

/* Human-readable name of a perm_status_t; never NULL. */
const char* perm_status_string(int status);

/* PERM_ABI_VERSION of the loaded library. */
int perm_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PERM_H */
