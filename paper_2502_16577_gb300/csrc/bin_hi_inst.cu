// Binary Ryser kernels for n = 33..63 (see binary.cuh).
#include "binary.cuh"
#include "kernels.h"

namespace permgpu {

template <int N>
static KernelEntry bin_hi_make() {
  return {reinterpret_cast<const void*>(&ryser_bin_kernel<N, 6>), BinLayout<N>::kBytes};
}

KernelEntry bin_hi_entry(int n) {
  switch (n) {
    case 33: return bin_hi_make<33>();
    case 34: return bin_hi_make<34>();
    case 35: return bin_hi_make<35>();
    case 36: return bin_hi_make<36>();
    case 37: return bin_hi_make<37>();
    case 38: return bin_hi_make<38>();
    case 39: return bin_hi_make<39>();
    case 40: return bin_hi_make<40>();
    case 41: return bin_hi_make<41>();
    case 42: return bin_hi_make<42>();
    case 43: return bin_hi_make<43>();
    case 44: return bin_hi_make<44>();
    case 45: return bin_hi_make<45>();
    case 46: return bin_hi_make<46>();
    case 47: return bin_hi_make<47>();
    case 48: return bin_hi_make<48>();
    case 49: return bin_hi_make<49>();
    case 50: return bin_hi_make<50>();
    case 51: return bin_hi_make<51>();
    case 52: return bin_hi_make<52>();
    case 53: return bin_hi_make<53>();
    case 54: return bin_hi_make<54>();
    case 55: return bin_hi_make<55>();
    case 56: return bin_hi_make<56>();
    case 57: return bin_hi_make<57>();
    case 58: return bin_hi_make<58>();
    case 59: return bin_hi_make<59>();
    case 60: return bin_hi_make<60>();
    case 61: return bin_hi_make<61>();
    case 62: return bin_hi_make<62>();
    case 63: return bin_hi_make<63>();
    default: return {nullptr, 0};
  }
}

}  // namespace permgpu
