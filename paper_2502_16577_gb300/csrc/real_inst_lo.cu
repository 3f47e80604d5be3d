// Real dense Ryser kernels for n = 1..24 (see real.cuh).
#include "real.cuh"
#include "kernels.h"

namespace permgpu {

template <int N>
static KernelEntry real_make() {
  return {reinterpret_cast<const void*>(&ryser_real_kernel<N>), RealLayout<N>::kBytes};
}

KernelEntry real_entry_lo(int n) {
  switch (n) {
    case 1: return real_make<1>();
    case 2: return real_make<2>();
    case 3: return real_make<3>();
    case 4: return real_make<4>();
    case 5: return real_make<5>();
    case 6: return real_make<6>();
    case 7: return real_make<7>();
    case 8: return real_make<8>();
    case 9: return real_make<9>();
    case 10: return real_make<10>();
    case 11: return real_make<11>();
    case 12: return real_make<12>();
    case 13: return real_make<13>();
    case 14: return real_make<14>();
    case 15: return real_make<15>();
    case 16: return real_make<16>();
    case 17: return real_make<17>();
    case 18: return real_make<18>();
    case 19: return real_make<19>();
    case 20: return real_make<20>();
    case 21: return real_make<21>();
    case 22: return real_make<22>();
    case 23: return real_make<23>();
    case 24: return real_make<24>();
    default: return {nullptr, 0};
  }
}

}  // namespace permgpu
