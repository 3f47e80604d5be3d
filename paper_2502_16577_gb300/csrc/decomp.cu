// Sparse preprocessing (Sec. 4): host-side graph work that turns one sparse
// permanent into a few smaller ones, evaluated by the GPU kernels.
//
//  1. Dulmage-Mendelsohn (Sec. 4.1).  A perfect matching M of the bipartite
//     row/column graph is found by augmenting paths (none: perm = 0).  With
//     every row contracted with its matched column, row i points to row k when
//     a_{i, M(k)} != 0; an entry a_ij (j != M(i)) lies on some perfect matching
//     iff i and the row matched to j are in the same strongly connected
//     component (Tarjan).  The other entries cannot contribute to any term of
//     Eq. 1 and are dropped, and what is left is a permuted block-diagonal
//     matrix: perm(A) = prod over components of perm(block).
//  2. Forbert-Marx (Sec. 4.2, Alg. 4).  Per block, the row or column with the
//     fewest nonzeros (transposing for a column, perm(A) = perm(A^T)) is
//     removed by the expansion of Eq. expand:
//       1 nonzero  alpha           -> alpha * perm(A without its row and column)
//       2 nonzeros alpha, beta     -> perm([alpha e + beta d | B])  (n-1)
//       3-4 nonzeros               -> perm(A with alpha, beta zeroed) + the
//                                     (n-1) matrix above
//     until every line of a matrix has more than four nonzeros.  The leaves
//     carry the products of the alphas as coefficients.
//  3. Every leaf of order >= 2 is evaluated on the GPU by the dense kernel
//     (density >= 30 %) or the sparse kernel (Alg. 2) otherwise, all
//     launches on one stream into one device array; the host adds
//     coefficient * leaf per block and multiplies the blocks in
//     double-double.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include <cuda_runtime.h>

#include "perm.h"

namespace {

struct Mat {
  int n = 0;
  std::vector<double> a;  // row-major n*n
  double& at(int i, int j) { return a[(size_t)i * n + j]; }
  double at(int i, int j) const { return a[(size_t)i * n + j]; }
};

struct Leaf {
  int block;
  double coef;
  Mat m;
};

struct hdd {
  double hi, lo;
};

hdd two_sum(double a, double b) {
  volatile double s = a + b;
  volatile double bv = s - a;
  double e = (a - (s - bv)) + (b - bv);
  return hdd{s, e};
}

hdd hdd_add(hdd x, hdd y) {
  hdd s = two_sum(x.hi, y.hi);
  double e = s.lo + x.lo + y.lo;
  return two_sum(s.hi, e);
}

hdd hdd_mul_d(hdd x, double b) {
  const double p = x.hi * b;
  const double e = fma(x.hi, b, -p);
  return two_sum(p, e + x.lo * b);
}

hdd hdd_mul(hdd x, hdd y) {
  const double p = x.hi * y.hi;
  const double e = fma(x.hi, y.hi, -p);
  return two_sum(p, e + x.hi * y.lo + x.lo * y.hi);
}

// ----------------------------------------------------------------- matching

bool augment(int i, const Mat& A, std::vector<int>& col_of, std::vector<int>& row_of, std::vector<char>& seen) {
  for (int j = 0; j < A.n; ++j) {
    if (A.at(i, j) == 0.0 || seen[j]) continue;
    seen[j] = 1;
    if (row_of[j] < 0 || augment(row_of[j], A, col_of, row_of, seen)) {
      row_of[j] = i;
      col_of[i] = j;
      return true;
    }
  }
  return false;
}

// Tarjan's strongly connected components (iterative) of the contracted row
// graph: i -> k iff a_{i, M(k)} != 0.
std::vector<int> scc_rows(const Mat& A, const std::vector<int>& col_of, const std::vector<int>& row_of) {
  const int n = A.n;
  std::vector<int> index(n, -1), low(n, 0), comp(n, -1), stack;
  std::vector<char> on(n, 0);
  int counter = 0, ncomp = 0;
  struct Frame {
    int v, next;
  };
  for (int s = 0; s < n; ++s) {
    if (index[s] >= 0) continue;
    std::vector<Frame> call{{s, 0}};
    index[s] = low[s] = counter++;
    stack.push_back(s);
    on[s] = 1;
    while (!call.empty()) {
      Frame& f = call.back();
      const int v = f.v;
      bool pushed = false;
      while (f.next < n) {
        const int j = f.next++;
        if (A.at(v, j) == 0.0) continue;
        const int k = row_of[j];  // column j belongs to row k's pair
        if (k == v) continue;
        if (index[k] < 0) {
          index[k] = low[k] = counter++;
          stack.push_back(k);
          on[k] = 1;
          call.push_back({k, 0});
          pushed = true;
          break;
        }
        if (on[k]) low[v] = std::min(low[v], index[k]);
      }
      if (pushed) continue;
      if (low[v] == index[v]) {
        while (true) {
          const int w = stack.back();
          stack.pop_back();
          on[w] = 0;
          comp[w] = ncomp;
          if (w == v) break;
        }
        ++ncomp;
      }
      call.pop_back();
      if (!call.empty()) {
        const int u = call.back().v;
        low[u] = std::min(low[u], low[v]);
      }
    }
  }
  (void)col_of;
  return comp;
}

// ------------------------------------------------------------ Forbert-Marx

Mat transpose(const Mat& A) {
  Mat T;
  T.n = A.n;
  T.a.resize(A.a.size());
  for (int i = 0; i < A.n; ++i)
    for (int j = 0; j < A.n; ++j) T.at(j, i) = A.at(i, j);
  return T;
}

Mat drop(const Mat& A, int r, int c) {
  Mat B;
  B.n = A.n - 1;
  B.a.resize((size_t)B.n * B.n);
  for (int i = 0, bi = 0; i < A.n; ++i) {
    if (i == r) continue;
    for (int j = 0, bj = 0; j < A.n; ++j) {
      if (j == c) continue;
      B.at(bi, bj++) = A.at(i, j);
    }
    ++bi;
  }
  return B;
}

// Eq. expand with row r = (alpha at j1, beta at j2, rest): the (n-1) x (n-1)
// matrix whose column j1 is alpha * col(j2) + beta * col(j1) (row r removed)
// and whose column j2 is removed.
Mat merge(const Mat& A, int r, int j1, int j2) {
  const double alpha = A.at(r, j1), beta = A.at(r, j2);
  Mat B;
  B.n = A.n - 1;
  B.a.resize((size_t)B.n * B.n);
  for (int i = 0, bi = 0; i < A.n; ++i) {
    if (i == r) continue;
    for (int j = 0, bj = 0; j < A.n; ++j) {
      if (j == j2) continue;
      B.at(bi, bj++) = (j == j1) ? fma(alpha, A.at(i, j2), beta * A.at(i, j1)) : A.at(i, j);
    }
    ++bi;
  }
  return B;
}

struct Decomp {
  int n = 0;
  int structurally_zero = 0;
  int nblocks = 0;
  int64_t removed = 0;
  int max_leaves = 0;
  int truncated = 0;
  Mat filtered;
  std::vector<Leaf> leaves;
};

void decomp_ryser(Decomp& d, Mat A, double coef, int block) {
  while (true) {
    if (coef == 0.0) return;
    if (A.n <= 1) {
      if (A.n == 1) coef *= A.at(0, 0);
      if (coef != 0.0) d.leaves.push_back({block, coef, Mat{}});
      return;
    }
    int best = A.n + 1, line = 0;
    bool col = false;
    for (int i = 0; i < A.n; ++i) {
      int c = 0;
      for (int j = 0; j < A.n; ++j) c += A.at(i, j) != 0.0;
      if (c < best) best = c, line = i, col = false;
    }
    for (int j = 0; j < A.n; ++j) {
      int c = 0;
      for (int i = 0; i < A.n; ++i) c += A.at(i, j) != 0.0;
      if (c < best) best = c, line = j, col = true;
    }
    if (best == 0) return;  // a zero line: this term is 0
    if (best > 4) break;
    if (col) A = transpose(A);
    int js[4], k = 0;
    for (int j = 0; j < A.n && k < 4; ++j)
      if (A.at(line, j) != 0.0) js[k++] = j;
    if (best == 1) {
      coef *= A.at(line, js[0]);
      A = drop(A, line, js[0]);
      continue;
    }
    if (best == 2) {
      A = merge(A, line, js[0], js[1]);
      continue;
    }
    if ((int)d.leaves.size() + 1 >= d.max_leaves) {
      d.truncated = 1;
      break;
    }
    Mat B = merge(A, line, js[0], js[1]);
    decomp_ryser(d, std::move(B), coef, block);
    A.at(line, js[0]) = 0.0;
    A.at(line, js[1]) = 0.0;
  }
  d.leaves.push_back({block, coef, std::move(A)});
}

int build(Decomp& d, int n, const int32_t* cptrs, const int32_t* rids, const double* cvals, int64_t nnz) {
  if (n < 0 || n > 63) return PERM_ERANGE;
  if (nnz < 0 || (n > 0 && (!cptrs || (nnz > 0 && (!rids || !cvals))))) return PERM_EINVAL;
  d.n = n;
  Mat A;
  A.n = n;
  A.a.assign((size_t)n * n, 0.0);
  if (n > 0) {
    if (cptrs[0] != 0 || cptrs[n] != nnz) return PERM_EINVAL;
    for (int j = 0; j < n; ++j) {
      if (cptrs[j + 1] < cptrs[j]) return PERM_EINVAL;
      for (int32_t p = cptrs[j]; p < cptrs[j + 1]; ++p) {
        const int i = rids[p];
        if (i < 0 || i >= n || (p > cptrs[j] && rids[p - 1] >= i)) return PERM_EINVAL;
        if (!isfinite(cvals[p])) return PERM_EINVAL;
        A.at(i, j) = cvals[p];
      }
    }
  }
  // a perfect matching of the nonzero pattern
  std::vector<int> col_of(n, -1), row_of(n, -1);
  for (int i = 0; i < n; ++i) {
    std::vector<char> seen(n, 0);
    if (!augment(i, A, col_of, row_of, seen)) {
      d.structurally_zero = 1;
      d.filtered = Mat{n, std::vector<double>((size_t)n * n, 0.0)};
      return PERM_OK;
    }
  }
  // fine Dulmage-Mendelsohn: drop the entries between components
  const std::vector<int> comp = scc_rows(A, col_of, row_of);
  int ncomp = 0;
  for (int c : comp) ncomp = std::max(ncomp, c + 1);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      if (A.at(i, j) != 0.0 && comp[i] != comp[row_of[j]]) {
        A.at(i, j) = 0.0;
        ++d.removed;
      }
  d.filtered = A;
  d.nblocks = ncomp;
  for (int c = 0; c < ncomp; ++c) {
    std::vector<int> rows;
    for (int i = 0; i < n; ++i)
      if (comp[i] == c) rows.push_back(i);
    Mat B;
    B.n = (int)rows.size();
    B.a.resize((size_t)B.n * B.n);
    for (int r = 0; r < B.n; ++r)
      for (int s = 0; s < B.n; ++s) B.at(r, s) = A.at(rows[r], col_of[rows[s]]);
    decomp_ryser(d, std::move(B), 1.0, c);
  }
  return PERM_OK;
}

}  // namespace

struct perm_decomp {
  Decomp d;
};

extern "C" {

int perm_decomp_create(perm_decomp** out, int n, const int32_t* cptrs, const int32_t* rids, const double* cvals,
                       int64_t nnz, int max_leaves) {
  if (!out) return PERM_EINVAL;
  *out = nullptr;
  perm_decomp* p = new (std::nothrow) perm_decomp;
  if (!p) return PERM_ENOMEM;
  p->d.max_leaves = max_leaves > 0 ? max_leaves : 4096;
  const int rc = build(p->d, n, cptrs, rids, cvals, nnz);
  if (rc != PERM_OK) {
    delete p;
    return rc;
  }
  *out = p;
  return PERM_OK;
}

int perm_decomp_info(const perm_decomp* p, perm_decomp_info_t* info) {
  if (!p || !info) return PERM_EINVAL;
  const Decomp& d = p->d;
  memset(info, 0, sizeof(*info));
  info->n = d.n;
  info->nblocks = d.nblocks;
  info->nleaves = (int)d.leaves.size();
  info->structurally_zero = d.structurally_zero;
  info->truncated = d.truncated;
  info->removed_nnz = d.removed;
  info->plain_steps = d.n > 0 ? ldexp(1.0, d.n - 1) : 0.0;
  for (const Leaf& l : d.leaves) {
    info->max_leaf_n = std::max(info->max_leaf_n, l.m.n);
    if (l.m.n > 0) info->leaf_steps += ldexp(1.0, l.m.n - 1);
  }
  return PERM_OK;
}

int perm_decomp_leaf(const perm_decomp* p, int index, int* n, int* block, double* coef, double* A) {
  if (!p || index < 0 || index >= (int)p->d.leaves.size()) return PERM_EINVAL;
  const Leaf& l = p->d.leaves[(size_t)index];
  if (n) *n = l.m.n;
  if (block) *block = l.block;
  if (coef) *coef = l.coef;
  if (A && l.m.n > 0) memcpy(A, l.m.a.data(), sizeof(double) * l.m.a.size());
  return PERM_OK;
}

int perm_decomp_filtered(const perm_decomp* p, double* A) {
  if (!p || !A) return PERM_EINVAL;
  if (p->d.n > 0) memcpy(A, p->d.filtered.a.data(), sizeof(double) * (size_t)p->d.n * p->d.n);
  return PERM_OK;
}

int perm_decomp_eval(perm_decomp* p, double* out, void* stream) {
  if (!p || !out) return PERM_EINVAL;
  const Decomp& d = p->d;
  if (d.n == 0) {
    *out = 1.0;
    return PERM_OK;
  }
  if (d.structurally_zero) {
    *out = 0.0;
    return PERM_OK;
  }
  // blocks whose leaves are all of order 0 (their value is the coefficient)
  // need no device at all
  bool any_gpu = false;
  for (const Leaf& l : d.leaves) any_gpu = any_gpu || l.m.n >= 2;
  if (!any_gpu) {
    std::vector<hdd> block(d.nblocks, hdd{0.0, 0.0});
    for (const Leaf& l : d.leaves) block[l.block] = hdd_add(block[l.block], hdd{l.coef, 0.0});
    hdd prod{1.0, 0.0};
    for (const hdd& x : block) prod = hdd_mul(prod, x);
    *out = prod.hi + prod.lo;
    return PERM_OK;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // Leaves of order 2..32 go to one batched launch (real batched plan);
  // larger ones get their own launch of the dense kernel (density >= 30 %)
  // or the sparse kernel.
  const size_t L = d.leaves.size();
  std::vector<size_t> off_dense(L, 0), off_cp(L, 0), off_nz(L, 0);
  std::vector<int64_t> leaf_nnz(L, 0), boff;
  std::vector<char> kind(L, 0);  // 1 batched, 2 dense, 3 sparse
  std::vector<int> bks, bidx(L, -1);
  size_t nd = 0, ncp = 0, nnz = 0, nb = 0;
  std::vector<double> hd, hv, hb;
  std::vector<int32_t> hcp, hr, blab;  // blab: row labels of the batched leaves
  bool repeats = false;
  for (size_t l = 0; l < L; ++l) {
    const Mat& m = d.leaves[l].m;
    if (m.n < 2) continue;
    size_t cnt = 0;
    for (double v : m.a) cnt += v != 0.0;
    leaf_nnz[l] = (int64_t)cnt;
    if (m.n <= 32) {
      kind[l] = 1;
      bidx[l] = (int)bks.size();
      bks.push_back(m.n);
      boff.push_back((int64_t)nb);
      hb.insert(hb.end(), m.a.begin(), m.a.end());
      nb += m.a.size();
      // equal rows (bitwise) share a label, so the batched plan sums them
      // over their multiplicities
      for (int i = 0; i < m.n; ++i) {
        int lab = i;
        for (int r = 0; r < i && lab == i; ++r)
          if (memcmp(&m.a[(size_t)r * m.n], &m.a[(size_t)i * m.n], sizeof(double) * m.n) == 0) lab = r;
        repeats |= lab != i;
        blab.push_back(lab);
      }
    } else if (cnt * 10 >= (size_t)m.n * m.n * 3) {
      kind[l] = 2;
      off_dense[l] = nd;
      hd.insert(hd.end(), m.a.begin(), m.a.end());
      nd += m.a.size();
    } else {
      kind[l] = 3;
      off_cp[l] = ncp;
      off_nz[l] = nnz;
      int32_t acc = 0;
      hcp.push_back(0);
      for (int j = 0; j < m.n; ++j) {
        for (int i = 0; i < m.n; ++i)
          if (m.at(i, j) != 0.0) {
            hr.push_back(i);
            hv.push_back(m.at(i, j));
            ++acc;
          }
        hcp.push_back(acc);
      }
      ncp += (size_t)m.n + 1;
      nnz += (size_t)acc;
    }
  }
  const size_t nbat = bks.size();
  const size_t bytes =
      sizeof(double) * (nd + nnz + L + nb + nbat) + sizeof(int32_t) * (ncp + nnz + L + nbat) + 64;
  void* ws = nullptr;
  if (cudaMalloc(&ws, bytes) != cudaSuccess) {
    cudaGetLastError();
    return PERM_ENOMEM;
  }
  double* dd_dense = static_cast<double*>(ws);
  double* dd_vals = dd_dense + nd;
  double* dd_out = dd_vals + nnz;
  double* dd_bat = dd_out + L;
  double* dd_bout = dd_bat + nb;
  int32_t* di_cp = reinterpret_cast<int32_t*>(dd_bout + nbat);
  int32_t* di_r = di_cp + ncp;
  int32_t* di_st = di_r + nnz;
  int32_t* di_bst = di_st + L;
  int rc = PERM_OK;
  auto cp = [&](void* dst, const void* src, size_t n) {
    if (rc == PERM_OK && n && cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, s) != cudaSuccess) rc = PERM_ECUDA;
  };
  cp(dd_dense, hd.data(), sizeof(double) * nd);
  cp(dd_vals, hv.data(), sizeof(double) * nnz);
  cp(di_cp, hcp.data(), sizeof(int32_t) * ncp);
  cp(di_r, hr.data(), sizeof(int32_t) * nnz);
  cp(dd_bat, hb.data(), sizeof(double) * nb);
  perm_batch_plan* plan = nullptr;
  if (rc == PERM_OK && nbat) {
    rc = repeats ? perm_batched_plan_create_labeled(&plan, PERM_F64, bks.data(), (int)nbat, dd_bat, boff.data(),
                                                    dd_bout, di_bst, blab.data())
                 : perm_batched_plan_create(&plan, PERM_F64, bks.data(), (int)nbat, dd_bat, boff.data(), dd_bout,
                                            di_bst);
    if (rc == PERM_OK) rc = perm_batched(plan, nullptr, nullptr, nullptr, stream);
  }
  for (size_t l = 0; l < L && rc == PERM_OK; ++l) {
    const Mat& m = d.leaves[l].m;
    if (kind[l] == 2)
      rc = perm(dd_dense + off_dense[l], m.n, PERM_F64, dd_out + l, di_st + l, stream);
    else if (kind[l] == 3)
      rc = perm_sparse(m.n, di_cp + off_cp[l], di_r + off_nz[l], dd_vals + off_nz[l], leaf_nnz[l], dd_out + l,
                       di_st + l, stream);
  }
  std::vector<double> vals(L, 1.0), bvals(nbat, 0.0);
  std::vector<int32_t> sts(L, 0), bsts(nbat, 0);
  auto back = [&](void* dst, const void* src, size_t n) {
    if (rc == PERM_OK && n && cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToHost, s) != cudaSuccess) rc = PERM_ECUDA;
  };
  back(vals.data(), dd_out, sizeof(double) * L);
  back(sts.data(), di_st, sizeof(int32_t) * L);
  back(bvals.data(), dd_bout, sizeof(double) * nbat);
  back(bsts.data(), di_bst, sizeof(int32_t) * nbat);
  if (cudaStreamSynchronize(s) != cudaSuccess && rc == PERM_OK) rc = PERM_ECUDA;
  if (plan) perm_batched_plan_destroy(plan);
  if (cudaFree(ws) != cudaSuccess && rc == PERM_OK) rc = PERM_ECUDA;
  if (rc != PERM_OK) {
    cudaGetLastError();
    return rc;
  }
  for (size_t l = 0; l < L; ++l) {
    if (kind[l] == 1) {
      sts[l] = bsts[bidx[l]];
      vals[l] = bvals[bidx[l]];
    }
  }
  std::vector<hdd> block(d.nblocks, hdd{0.0, 0.0});
  for (size_t l = 0; l < L; ++l) {
    const Mat& m = d.leaves[l].m;
    double v = 1.0;
    if (m.n >= 2) {
      if (sts[l] != PERM_OK) return sts[l];
      v = vals[l];
    }
    block[d.leaves[l].block] = hdd_add(block[d.leaves[l].block], hdd_mul_d(hdd{v, 0.0}, d.leaves[l].coef));
  }
  hdd prod{1.0, 0.0};
  for (const hdd& x : block) prod = hdd_mul(prod, x);
  *out = prod.hi + prod.lo;
  return PERM_OK;
}

void perm_decomp_destroy(perm_decomp* p) { delete p; }

int perm_sparse_decomp(int n, const int32_t* cptrs, const int32_t* rids, const double* cvals, int64_t nnz,
                       double* out, perm_decomp_info_t* info, void* stream) {
  perm_decomp* p = nullptr;
  int rc = perm_decomp_create(&p, n, cptrs, rids, cvals, nnz, 0);
  if (rc != PERM_OK) return rc;
  if (info) perm_decomp_info(p, info);
  rc = perm_decomp_eval(p, out, stream);
  perm_decomp_destroy(p);
  return rc;
}

}  // extern "C"
