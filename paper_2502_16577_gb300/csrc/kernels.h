// Instantiation tables of the dense kernels: one translation unit per range of
// n so that the 63 compile-time sizes build in parallel.
#pragma once
#include <stddef.h>
#include <stdint.h>

namespace permgpu {

struct KernelEntry {
  const void* fn;          // __global__ function
  size_t smem;             // dynamic shared memory in bytes
  int chunks_per_warp = 32;  // chunks one warp walks at a time (lanes per chunk = 32 / this)
};

KernelEntry real_entry_lo(int n);   // n = 1..24
KernelEntry real_entry_mid(int n);  // n = 25..44
KernelEntry real_entry_hi(int n);   // n = 45..63
KernelEntry bin_lo_entry(int n);    // n = 1..32
KernelEntry bin_hi_entry(int n);    // n = 33..63
KernelEntry cplx_lo_entry(int n);   // n = 1..24
KernelEntry cplx_hi_entry(int n);   // n = 25..63
KernelEntry realx_entry_lo(int n);  // n = 1..32, extended products
KernelEntry realx_entry_hi(int n);  // n = 33..63

// Device view of the word registered with perm_set_abort_word, or null (api.cu).
const volatile uint32_t* current_abort_word();

// Time budget of new sweeps in nanoseconds, 0 for none (perm_set_time_budget, api.cu).
uint64_t current_time_budget();

// Chunk exponent of a launch over nsteps Gray steps (api.cu).
int plan_chunk_exponent(int n, uint64_t nsteps, int warps_resident);

// Launch shape of a dense sweep over [g_begin, g_end): grid, chunk exponent
// and the visited chunks (api.cu; every dense entry point uses it).
struct RyserLaunch {
  int grid = 0, c = 0;
  uint64_t k_begin = 0, nchunks = 0;
};
int plan_ryser_launch(const KernelEntry& ke, int n, uint64_t g_begin, uint64_t g_end, RyserLaunch& L);

}  // namespace permgpu
