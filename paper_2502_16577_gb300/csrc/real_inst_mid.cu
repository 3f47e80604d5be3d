// Real dense Ryser kernels for n = 25..44 (see real.cuh).
#include "real.cuh"
#include "kernels.h"

namespace permgpu {

template <int N>
static KernelEntry real_make() {
  return {reinterpret_cast<const void*>(&ryser_real_kernel<N>), RealLayout<N>::kBytes};
}

KernelEntry real_entry_mid(int n) {
  switch (n) {
    case 25: return real_make<25>();
    case 26: return real_make<26>();
    case 27: return real_make<27>();
    case 28: return real_make<28>();
    case 29: return real_make<29>();
    case 30: return real_make<30>();
    case 31: return real_make<31>();
    case 32: return real_make<32>();
    case 33: return real_make<33>();
    case 34: return real_make<34>();
    case 35: return real_make<35>();
    case 36: return real_make<36>();
    case 37: return real_make<37>();
    case 38: return real_make<38>();
    case 39: return real_make<39>();
    case 40: return real_make<40>();
    case 41: return real_make<41>();
    case 42: return real_make<42>();
    case 43: return real_make<43>();
    case 44: return real_make<44>();
    default: return {nullptr, 0};
  }
}

}  // namespace permgpu
