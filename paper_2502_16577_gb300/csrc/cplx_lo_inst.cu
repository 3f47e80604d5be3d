// Complex Ryser kernels for n = 1..24 (see complex.cuh).
#include "complex.cuh"
#include "kernels.h"

namespace permgpu {

template <int N>
static KernelEntry cplx_lo_make() {
  // two lanes per chunk from n = 16 on (register pressure of the complex rows)
  if (N >= 16) return {reinterpret_cast<const void*>(&ryser_cplx2_kernel<N>), CplxLayout<N>::kBytes, 16};
  return {reinterpret_cast<const void*>(&ryser_cplx_kernel<N>), CplxLayout<N>::kBytes, 32};
}

KernelEntry cplx_lo_entry(int n) {
  switch (n) {
    case 1: return cplx_lo_make<1>();
    case 2: return cplx_lo_make<2>();
    case 3: return cplx_lo_make<3>();
    case 4: return cplx_lo_make<4>();
    case 5: return cplx_lo_make<5>();
    case 6: return cplx_lo_make<6>();
    case 7: return cplx_lo_make<7>();
    case 8: return cplx_lo_make<8>();
    case 9: return cplx_lo_make<9>();
    case 10: return cplx_lo_make<10>();
    case 11: return cplx_lo_make<11>();
    case 12: return cplx_lo_make<12>();
    case 13: return cplx_lo_make<13>();
    case 14: return cplx_lo_make<14>();
    case 15: return cplx_lo_make<15>();
    case 16: return cplx_lo_make<16>();
    case 17: return cplx_lo_make<17>();
    case 18: return cplx_lo_make<18>();
    case 19: return cplx_lo_make<19>();
    case 20: return cplx_lo_make<20>();
    case 21: return cplx_lo_make<21>();
    case 22: return cplx_lo_make<22>();
    case 23: return cplx_lo_make<23>();
    case 24: return cplx_lo_make<24>();
    default: return {nullptr, 0};
  }
}

}  // namespace permgpu
