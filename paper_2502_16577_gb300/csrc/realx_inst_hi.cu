// Extended-product real Ryser kernels for n = 33..63 (see realx.cuh).
#include <utility>

#include "kernels.h"
#include "realx.cuh"

namespace permgpu {

template <int N>
static KernelEntry realx_make() {
  return {reinterpret_cast<const void*>(&ryser_realx_kernel<N>), RealLayout<N>::kBytes};
}

template <int... I>
static KernelEntry realx_pick(int n, std::integer_sequence<int, I...>) {
  KernelEntry e{nullptr, 0};
  ((n == I + 33 ? (e = realx_make<I + 33>(), 0) : 0), ...);
  return e;
}

KernelEntry realx_entry_hi(int n) { return realx_pick(n, std::make_integer_sequence<int, 31>{}); }

}  // namespace permgpu
