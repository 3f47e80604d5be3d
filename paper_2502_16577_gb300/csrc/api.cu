// C ABI of libperm.so (include/perm.h): argument checks, launch planning,
// scratch memory and the host-side combination of range partials.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <tuple>

#include "common.cuh"
#include "kernels.h"

namespace permgpu {

// ----------------------------------------------------------- device facts

struct DeviceFacts {
  int sms = 0;
};

static int current_device_facts(DeviceFacts& f) {
  static std::mutex mu;
  static DeviceFacts cache[64];
  static bool have[64] = {false};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return PERM_ECUDA;
  std::lock_guard<std::mutex> lock(mu);
  if (!have[dev]) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PERM_ECUDA;
    cache[dev].sms = sms;
    have[dev] = true;
  }
  f = cache[dev];
  return PERM_OK;
}

// Blocks per SM of a kernel (after raising its dynamic shared-memory limit),
// queried once per device, kernel and shared-memory size instead of on every
// launch.
static int blocks_per_sm(const KernelEntry& ke) {
  static std::mutex mu;
  static std::map<std::tuple<int, const void*, size_t>, int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  const auto key = std::make_tuple(dev, ke.fn, ke.smem);
  std::lock_guard<std::mutex> lock(mu);
  const auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  if (ke.smem > 48 * 1024) {
    if (cudaFuncSetAttribute(ke.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ke.smem) != cudaSuccess)
      return -1;
  }
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ke.fn, kBlock, ke.smem) != cudaSuccess) return -1;
  if (nb > 0) cache.emplace(key, nb);
  return nb;
}

static int ceil_log2_u64(uint64_t v) {
  int r = 0;
  while ((1ull << r) < v) ++r;
  return r;
}

static int floor_log2_u64(uint64_t v) {
  int r = -1;
  while (v) {
    v >>= 1;
    ++r;
  }
  return r;
}

// ------------------------------------------------- cancellation, time budget

static std::atomic<const volatile uint32_t*> g_abort_word{nullptr};
static std::atomic<uint64_t> g_budget_ns{0};

const volatile uint32_t* current_abort_word() { return g_abort_word.load(std::memory_order_acquire); }

uint64_t current_time_budget() { return g_budget_ns.load(std::memory_order_acquire); }

// Chunk exponent c: aligned chunks of 2^c steps (Sec. 3.1.1).  Aim for at
// least 64 warp-groups of 32 chunks per resident warp (tail below ~1.6%), but
// keep 2^c >= 4n so that starting a chunk (at most n(n-c) adds) stays small
// against its 2^c steps of n multiplies.
int plan_chunk_exponent(int n, uint64_t nsteps, int warps_resident) {
  int cmax = n - 1 < 30 ? n - 1 : 30;
  if (cmax < 0) cmax = 0;
  int cmin = ceil_log2_u64((uint64_t)n) + 2;
  if (cmin > cmax) cmin = cmax;
  uint64_t want = 32ull * 64ull * (uint64_t)(warps_resident > 0 ? warps_resident : 1);
  int c = nsteps > want ? floor_log2_u64(nsteps / want) : 0;
  if (c < cmin) c = cmin;
  if (c > cmax) c = cmax;
  return c;
}

int plan_ryser_launch(const KernelEntry& ke, int n, uint64_t g_begin, uint64_t g_end, RyserLaunch& L) {
  if (!ke.fn) return PERM_EINVAL;
  DeviceFacts df;
  int rc = current_device_facts(df);
  if (rc) return rc;
  int nb = blocks_per_sm(ke);
  if (nb <= 0) return PERM_ECUDA;
  const int grid_full = df.sms * nb;
  L.c = plan_chunk_exponent(n, g_end - g_begin, grid_full * kWarps);
  L.k_begin = g_begin >> L.c;
  const uint64_t k_end = (g_end + (1ull << L.c) - 1) >> L.c;
  L.nchunks = g_end > g_begin ? k_end - L.k_begin : 0;
  const uint64_t cpw = (uint64_t)(ke.chunks_per_warp > 0 ? ke.chunks_per_warp : 32);
  const uint64_t groups = (L.nchunks + cpw - 1) / cpw;
  const uint64_t need = (groups + kWarps - 1) / kWarps;
  L.grid = (int)(need < (uint64_t)grid_full ? (need > 0 ? need : 1) : grid_full);
  return PERM_OK;
}

// One Ryser launch over [g_begin, g_end): scratch from the stream-ordered
// allocator, arrival counter zeroed, kernel, scratch released.
static int launch_ryser(const KernelEntry& ke, const void* A, int n, uint64_t g_begin, uint64_t g_end, int mode,
                        void* out, int32_t* status, cudaStream_t s, size_t part_bytes) {
  RyserLaunch L;
  int rc = plan_ryser_launch(ke, n, g_begin, g_end, L);
  if (rc) return rc;
  const int grid = L.grid, c = L.c;
  const uint64_t k_begin = L.k_begin, nchunks = L.nchunks;

  size_t bytes = part_bytes * (size_t)grid + 16;
  void* ws = nullptr;
  if (cudaMallocAsync(&ws, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return PERM_ENOMEM;
  }
  unsigned int* counter = reinterpret_cast<unsigned int*>(static_cast<char*>(ws) + part_bytes * (size_t)grid);
  if (cudaMemsetAsync(counter, 0, 2 * sizeof(unsigned int), s) != cudaSuccess) {
    cudaFreeAsync(ws, s);
    return PERM_ECUDA;
  }
  RyserArgs args;
  memset(&args, 0, sizeof(args));
  args.A = A;
  args.n = n;
  args.c = c;
  args.mode = mode;
  args.g_begin = g_begin;
  args.g_end = g_end;
  args.k_begin = k_begin;
  args.nchunks = nchunks;
  args.part = ws;
  args.counter = counter;
  args.out = out;
  args.status = status;
  args.abort_word = current_abort_word();
  args.aborted = counter + 1;
  args.budget_ns = current_time_budget();
  void* params[] = {&args};
  cudaError_t e = cudaLaunchKernel(ke.fn, dim3(grid), dim3(kBlock), params, ke.smem, s);
  cudaError_t f = cudaFreeAsync(ws, s);
  if (e != cudaSuccess || f != cudaSuccess) {
    cudaGetLastError();
    return PERM_ECUDA;
  }
  return PERM_OK;
}

static KernelEntry dense_entry(int type, int n) {
  switch (type) {
    case PERM_F64:
      if (n <= 24) return real_entry_lo(n);
      if (n <= 44) return real_entry_mid(n);
      return real_entry_hi(n);
    case PERM_C128:
      return n <= 24 ? cplx_lo_entry(n) : cplx_hi_entry(n);
    case PERM_BIN:
      return n <= 32 ? bin_lo_entry(n) : bin_hi_entry(n);
    case PERM_F64X:
      return n <= 32 ? realx_entry_lo(n) : realx_entry_hi(n);
    default:
      return {nullptr, 0};
  }
}

static size_t partial_bytes(int type) {
  switch (type) {
    case PERM_F64:
    case PERM_F64X: return sizeof(dd);
    case PERM_C128: return 2 * sizeof(dd);
    default: return 8 * sizeof(uint32_t);
  }
}

// perm of the 0 x 0 matrix, and empty ranges, need no kernel of their own.
__global__ void write_trivial_kernel(int type, int mode, void* out, int32_t* status) {
  if (threadIdx.x != 0) return;
  if (type == PERM_F64) {
    double* o = static_cast<double*>(out);
    if (mode == 0) o[0] = 1.0;
    else o[0] = o[1] = 0.0;
  } else if (type == PERM_C128 || type == PERM_F64X) {
    double* o = static_cast<double*>(out);
    if (mode == 0) { o[0] = 1.0; o[1] = 0.0; }
    else if (type == PERM_C128) o[0] = o[1] = o[2] = o[3] = 0.0;
    else o[0] = o[1] = 0.0;
  } else {
    uint64_t* o = static_cast<uint64_t*>(out);
    if (mode == 0) { o[0] = 1; o[1] = 0; }
    else o[0] = o[1] = o[2] = 0;
  }
  if (status) *status = PERM_OK;
}

static int dispatch(const void* A, int n, int type, uint64_t g0, uint64_t g1, int mode, void* out, int32_t* status,
                    void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n == 0) {
    write_trivial_kernel<<<1, 32, 0, s>>>(type, mode, out, status);
    return cudaGetLastError() == cudaSuccess ? PERM_OK : PERM_ECUDA;
  }
  KernelEntry ke = dense_entry(type, n);
  if (!ke.fn) return PERM_EINVAL;
  return launch_ryser(ke, A, n, g0, g1, mode, out, status, s, partial_bytes(type));
}

// ------------------------------------------------------- host double-double

struct hdd {
  double hi, lo;
};

static hdd hdd_add(hdd a, hdd b) {
  volatile double s = a.hi + b.hi;
  volatile double bv = s - a.hi;
  double e = (a.hi - (s - bv)) + (b.hi - bv);
  e += a.lo + b.lo;
  volatile double h = s + e;
  hdd r;
  r.lo = e - (h - s);
  r.hi = h;
  return r;
}

}  // namespace permgpu

using namespace permgpu;

extern "C" {

int perm_abi_version(void) { return PERM_ABI_VERSION; }

int perm_set_abort_word(volatile uint32_t* host_mapped) {
  if (!host_mapped) {
    g_abort_word.store(nullptr, std::memory_order_release);
    return PERM_OK;
  }
  void* dev = nullptr;
  if (cudaHostGetDevicePointer(&dev, const_cast<uint32_t*>(host_mapped), 0) != cudaSuccess) {
    cudaGetLastError();
    return PERM_EINVAL;  // not page-locked mapped host memory
  }
  g_abort_word.store(static_cast<const volatile uint32_t*>(dev), std::memory_order_release);
  return PERM_OK;
}

int perm_set_time_budget(uint64_t nanoseconds) {
  g_budget_ns.store(nanoseconds, std::memory_order_release);
  return PERM_OK;
}

int perm_abort_word_alloc(volatile uint32_t** host_word) {
  if (!host_word) return PERM_EINVAL;
  void* p = nullptr;
  if (cudaHostAlloc(&p, sizeof(uint32_t), cudaHostAllocMapped) != cudaSuccess) {
    cudaGetLastError();
    return PERM_ENOMEM;
  }
  *static_cast<volatile uint32_t*>(p) = 0u;
  *host_word = static_cast<volatile uint32_t*>(p);
  return PERM_OK;
}

int perm_abort_word_free(volatile uint32_t* host_word) {
  if (!host_word) return PERM_OK;
  if (g_abort_word.load() != nullptr) {
    void* dev = nullptr;
    if (cudaHostGetDevicePointer(&dev, const_cast<uint32_t*>(host_word), 0) == cudaSuccess &&
        dev == (const void*)g_abort_word.load())
      g_abort_word.store(nullptr);
  }
  return cudaFreeHost(const_cast<uint32_t*>(host_word)) == cudaSuccess ? PERM_OK : PERM_ECUDA;
}

const char* perm_status_string(int status) {
  switch (status) {
    case PERM_OK: return "PERM_OK";
    case PERM_EINVAL: return "PERM_EINVAL: invalid argument or matrix entry";
    case PERM_ERANGE: return "PERM_ERANGE: size, range or binary64 exponent out of range";
    case PERM_EOVERFLOW: return "PERM_EOVERFLOW: the permanent may not fit the output";
    case PERM_ECUDA: return "PERM_ECUDA: a CUDA call failed";
    case PERM_ENOMEM: return "PERM_ENOMEM: scratch allocation failed";
    case PERM_EABORTED: return "PERM_EABORTED: stopped by the registered abort word";
    case PERM_ETIMEOUT: return "PERM_ETIMEOUT: stopped when the time budget ran out";
    default: return "unknown perm status";
  }
}

static int check_common(const void* A, int n, int type, const void* out) {
  if (type != PERM_F64 && type != PERM_C128 && type != PERM_BIN && type != PERM_F64X) return PERM_EINVAL;
  if (n < 0 || n > PERM_NMAX) return PERM_ERANGE;
  if (!out || (n > 0 && !A)) return PERM_EINVAL;
  return PERM_OK;
}

int perm(const void* A, int n, int type, void* out, int32_t* status, void* stream) {
  int rc = check_common(A, n, type, out);
  if (rc) return rc;
  uint64_t N = n > 0 ? 1ull << (n - 1) : 0;
  return dispatch(A, n, type, 0, N, 0, out, status, stream);
}

int perm_range(const void* A, int n, int type, uint64_t g_begin, uint64_t g_end, void* partial, int32_t* status,
               void* stream) {
  int rc = check_common(A, n, type, partial);
  if (rc) return rc;
  uint64_t N = n > 0 ? 1ull << (n - 1) : 0;
  if (g_begin > g_end || g_end > N) return PERM_ERANGE;
  if (n == 0 || g_begin == g_end) {
    write_trivial_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(type, 1, partial, status);
    return cudaGetLastError() == cudaSuccess ? PERM_OK : PERM_ECUDA;
  }
  return dispatch(A, n, type, g_begin, g_end, 1, partial, status, stream);
}

int perm_combine(int type, int n, const void* partials, int count, void* out) {
  if (n < 0 || n > PERM_NMAX) return PERM_ERANGE;
  if (!out || count < 0 || (count > 0 && !partials)) return PERM_EINVAL;
  if (type == PERM_F64 || type == PERM_C128) {
    int w = type == PERM_F64 ? 1 : 2;
    const double* p = static_cast<const double*>(partials);
    double* o = static_cast<double*>(out);
    if (n == 0) {
      o[0] = 1.0;
      if (w == 2) o[1] = 0.0;
      return PERM_OK;
    }
    double f = (n & 1) ? 2.0 : -2.0;
    for (int c = 0; c < w; ++c) {
      hdd acc = {0.0, 0.0};
      for (int i = 0; i < count; ++i) acc = hdd_add(acc, hdd{p[(size_t)i * 2 * w + 2 * c], p[(size_t)i * 2 * w + 2 * c + 1]});
      o[c] = (acc.hi + acc.lo) * f;
    }
    return PERM_OK;
  }
  if (type == PERM_F64X) {
    const double* p = static_cast<const double*>(partials);
    double* o = static_cast<double*>(out);
    if (n == 0) {
      o[0] = 1.0;
      o[1] = 0.0;
      return PERM_OK;
    }
    hdd acc = {0.0, 0.0};
    for (int i = 0; i < count; ++i) acc = hdd_add(acc, hdd{p[2 * (size_t)i], p[2 * (size_t)i + 1]});
    const double f = (n & 1) ? 2.0 : -2.0;  // exact on both words
    o[0] = acc.hi * f;
    o[1] = acc.lo * f;
    return PERM_OK;
  }
  if (type == PERM_BIN) {
    const uint64_t* p = static_cast<const uint64_t*>(partials);
    uint64_t* o = static_cast<uint64_t*>(out);
    if (n == 0) {
      o[0] = 1;
      o[1] = 0;
      return PERM_OK;
    }
    unsigned __int128 lo = 0;
    uint64_t hi = 0;
    for (int i = 0; i < count; ++i) {
      unsigned __int128 add = ((unsigned __int128)p[3 * (size_t)i + 1] << 64) | p[3 * (size_t)i];
      unsigned __int128 s = lo + add;
      hi += p[3 * (size_t)i + 2] + (s < lo ? 1u : 0u);
      lo = s;
    }
    // sum = (-1)^(n-1) 2^(n-1) perm(A)  (mod 2^192)
    if ((n - 1) & 1) {  // negate mod 2^192
      lo = ~lo;
      hi = ~hi;
      lo += 1;
      if (lo == 0) hi += 1;
    }
    int sh = n - 1;
    if (sh > 0) {
      unsigned __int128 mask = ((unsigned __int128)1 << sh) - 1;
      if (lo & mask) return PERM_EINVAL;
      lo = (lo >> sh) | ((unsigned __int128)hi << (128 - sh));
      hi >>= sh;
    }
    if (hi != 0) return PERM_EOVERFLOW;
    o[0] = (uint64_t)lo;
    o[1] = (uint64_t)(lo >> 64);
    return PERM_OK;
  }
  return PERM_EINVAL;
}

int perm_host(const void* A_host, int n, int type, void* out_host, void* stream) {
  int rc = check_common(A_host, n, type, out_host);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  size_t elem = (type == PERM_F64 || type == PERM_F64X) ? sizeof(double)
                : type == PERM_C128                      ? 2 * sizeof(double)
                                                         : sizeof(uint8_t);
  size_t in_bytes = elem * (size_t)n * (size_t)n;
  size_t out_bytes = type == PERM_F64 ? sizeof(double) : 2 * sizeof(uint64_t);
  void* dA = nullptr;
  void* dOut = nullptr;
  if (cudaMallocAsync(&dA, in_bytes + 256 + out_bytes + 16, s) != cudaSuccess) {
    cudaGetLastError();
    return PERM_ENOMEM;
  }
  dOut = static_cast<char*>(dA) + ((in_bytes + 255) & ~(size_t)255);
  int32_t* dStatus = reinterpret_cast<int32_t*>(static_cast<char*>(dOut) + out_bytes);
  int32_t hstatus = PERM_OK;
  rc = PERM_OK;
  if (in_bytes && cudaMemcpyAsync(dA, A_host, in_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) rc = PERM_ECUDA;
  if (!rc) rc = perm(dA, n, type, dOut, dStatus, stream);
  if (!rc && cudaMemcpyAsync(out_host, dOut, out_bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) rc = PERM_ECUDA;
  if (!rc && cudaMemcpyAsync(&hstatus, dStatus, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    rc = PERM_ECUDA;
  cudaFreeAsync(dA, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) rc = PERM_ECUDA;
  if (rc) {
    cudaGetLastError();
    return rc;
  }
  return hstatus;
}

}  // extern "C"
