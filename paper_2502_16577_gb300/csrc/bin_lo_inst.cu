// Binary Ryser kernels for n = 1..32 (see binary.cuh).
#include "binary.cuh"
#include "kernels.h"

namespace permgpu {

template <int N>
static KernelEntry bin_lo_make() {
  return {reinterpret_cast<const void*>(&ryser_bin_kernel<N, 6>), BinLayout<N>::kBytes};
}

KernelEntry bin_lo_entry(int n) {
  switch (n) {
    case 1: return bin_lo_make<1>();
    case 2: return bin_lo_make<2>();
    case 3: return bin_lo_make<3>();
    case 4: return bin_lo_make<4>();
    case 5: return bin_lo_make<5>();
    case 6: return bin_lo_make<6>();
    case 7: return bin_lo_make<7>();
    case 8: return bin_lo_make<8>();
    case 9: return bin_lo_make<9>();
    case 10: return bin_lo_make<10>();
    case 11: return bin_lo_make<11>();
    case 12: return bin_lo_make<12>();
    case 13: return bin_lo_make<13>();
    case 14: return bin_lo_make<14>();
    case 15: return bin_lo_make<15>();
    case 16: return bin_lo_make<16>();
    case 17: return bin_lo_make<17>();
    case 18: return bin_lo_make<18>();
    case 19: return bin_lo_make<19>();
    case 20: return bin_lo_make<20>();
    case 21: return bin_lo_make<21>();
    case 22: return bin_lo_make<22>();
    case 23: return bin_lo_make<23>();
    case 24: return bin_lo_make<24>();
    case 25: return bin_lo_make<25>();
    case 26: return bin_lo_make<26>();
    case 27: return bin_lo_make<27>();
    case 28: return bin_lo_make<28>();
    case 29: return bin_lo_make<29>();
    case 30: return bin_lo_make<30>();
    case 31: return bin_lo_make<31>();
    case 32: return bin_lo_make<32>();
    default: return {nullptr, 0};
  }
}

}  // namespace permgpu
