// Real dense Ryser kernels for n = 45..63 (see real.cuh).
#include "real.cuh"
#include "kernels.h"

namespace permgpu {

template <int N>
static KernelEntry real_make() {
  return {reinterpret_cast<const void*>(&ryser_real_kernel<N>), RealLayout<N>::kBytes};
}

KernelEntry real_entry_hi(int n) {
  switch (n) {
    case 45: return real_make<45>();
    case 46: return real_make<46>();
    case 47: return real_make<47>();
    case 48: return real_make<48>();
    case 49: return real_make<49>();
    case 50: return real_make<50>();
    case 51: return real_make<51>();
    case 52: return real_make<52>();
    case 53: return real_make<53>();
    case 54: return real_make<54>();
    case 55: return real_make<55>();
    case 56: return real_make<56>();
    case 57: return real_make<57>();
    case 58: return real_make<58>();
    case 59: return real_make<59>();
    case 60: return real_make<60>();
    case 61: return real_make<61>();
    case 62: return real_make<62>();
    case 63: return real_make<63>();
    default: return {nullptr, 0};
  }
}

}  // namespace permgpu
