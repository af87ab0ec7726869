// Kernel instantiations for the D3Q19 lattice (fused step and its adjoint).
#include "dispatch.cuh"

namespace lbf {
KernelInfo forward_kernel_q19(int storage, bool mask, bool two, bool tma) {
  return forward_kernel<D3Q19>(storage, mask, two, tma);
}
KernelInfo adjoint_kernel_q19(int storage, bool mask) { return adjoint_kernel<D3Q19>(storage, mask); }
}  // namespace lbf
