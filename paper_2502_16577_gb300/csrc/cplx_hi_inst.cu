// Complex Ryser kernels for n = 25..63 (see complex.cuh).
#include "complex.cuh"
#include "kernels.h"

namespace permgpu {

template <int N>
static KernelEntry cplx_hi_make() {
  // two lanes per chunk from n = 16 on (register pressure of the complex rows)
  if (N >= 16) return {reinterpret_cast<const void*>(&ryser_cplx2_kernel<N>), CplxLayout<N>::kBytes, 16};
  return {reinterpret_cast<const void*>(&ryser_cplx_kernel<N>), CplxLayout<N>::kBytes, 32};
}

KernelEntry cplx_hi_entry(int n) {
  switch (n) {
    case 25: return cplx_hi_make<25>();
    case 26: return cplx_hi_make<26>();
    case 27: return cplx_hi_make<27>();
    case 28: return cplx_hi_make<28>();
    case 29: return cplx_hi_make<29>();
    case 30: return cplx_hi_make<30>();
    case 31: return cplx_hi_make<31>();
    case 32: return cplx_hi_make<32>();
    case 33: return cplx_hi_make<33>();
    case 34: return cplx_hi_make<34>();
    case 35: return cplx_hi_make<35>();
    case 36: return cplx_hi_make<36>();
    case 37: return cplx_hi_make<37>();
    case 38: return cplx_hi_make<38>();
    case 39: return cplx_hi_make<39>();
    case 40: return cplx_hi_make<40>();
    case 41: return cplx_hi_make<41>();
    case 42: return cplx_hi_make<42>();
    case 43: return cplx_hi_make<43>();
    case 44: return cplx_hi_make<44>();
    case 45: return cplx_hi_make<45>();
    case 46: return cplx_hi_make<46>();
    case 47: return cplx_hi_make<47>();
    case 48: return cplx_hi_make<48>();
    case 49: return cplx_hi_make<49>();
    case 50: return cplx_hi_make<50>();
    case 51: return cplx_hi_make<51>();
    case 52: return cplx_hi_make<52>();
    case 53: return cplx_hi_make<53>();
    case 54: return cplx_hi_make<54>();
    case 55: return cplx_hi_make<55>();
    case 56: return cplx_hi_make<56>();
    case 57: return cplx_hi_make<57>();
    case 58: return cplx_hi_make<58>();
    case 59: return cplx_hi_make<59>();
    case 60: return cplx_hi_make<60>();
    case 61: return cplx_hi_make<61>();
    case 62: return cplx_hi_make<62>();
    case 63: return cplx_hi_make<63>();
    default: return {nullptr, 0};
  }
}

}  // namespace permgpu
