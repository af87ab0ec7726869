// Kernel instantiations of one (lattice, storage) pair: the fused step in every force / mask / TMA
// variant (30-column tiles, and line-aligned 32-column tiles with TMA stores for FP32 and 16-bit
// storage) and, for FP64 and FP32 storage, its adjoint. The build compiles this file once per pair
// with LBF_TU_LATTICE (19, 27 or 127 = D3Q27h) and LBF_TU_STORAGE (0 FP64, 1 FP32, 2 FP16, 3 BF16) defined.
#include "dispatch.cuh"

#if !defined(LBF_TU_LATTICE) || !defined(LBF_TU_STORAGE)
#error "compile kernels.cu with -DLBF_TU_LATTICE=19|27|127 -DLBF_TU_STORAGE=0..3"
#endif

namespace lbf {
namespace {
#if LBF_TU_LATTICE == 19
using TuL = D3Q19;
#elif LBF_TU_LATTICE == 27
using TuL = D3Q27;
#elif LBF_TU_LATTICE == 127
using TuL = D3Q27H;
#else
#error "LBF_TU_LATTICE must be 19, 27 or 127"
#endif
#if LBF_TU_STORAGE == 0
using TuS = double;
#elif LBF_TU_STORAGE == 1
using TuS = float;
#elif LBF_TU_STORAGE == 2
using TuS = __half;
#elif LBF_TU_STORAGE == 3
using TuS = __nv_bfloat16;
#else
#error "LBF_TU_STORAGE must be 0..3"
#endif
}  // namespace

#define LBF_CAT2(a, b, c, d) a##b##c##d
#define LBF_CAT(a, b, c, d) LBF_CAT2(a, b, c, d)

KernelInfo LBF_CAT(forward_kernel_q, LBF_TU_LATTICE, _s, LBF_TU_STORAGE)(bool mask, int two, bool field, bool tma,
                                                                         bool nearest) {
  return forward_kernel_ls<TuL, TuS>(mask, two, field, tma, nearest);
}

KernelInfo LBF_CAT(aligned_kernel_q, LBF_TU_LATTICE, _s, LBF_TU_STORAGE)(bool mask, bool field, bool nearest) {
  return aligned_kernel_ls<TuL, TuS>(mask, field, nearest);
}

PopKernels LBF_CAT(pop_kernels_q, LBF_TU_LATTICE, _s, LBF_TU_STORAGE)(bool mask, bool field) {
#if LBF_TU_LATTICE == 127
  (void)mask;
  (void)field;
  return PopKernels{nullptr, nullptr, nullptr};  // the population kernels collide at second order
#else
  return pop_kernels_ls<TuL, TuS>(mask, field);
#endif
}

KernelInfo LBF_CAT(adjoint_kernel_q, LBF_TU_LATTICE, _s, LBF_TU_STORAGE)(bool mask) {
#if LBF_TU_STORAGE <= 1 && LBF_TU_LATTICE != 127
  return mask ? adj_info<TuL, TuS, true>() : adj_info<TuL, TuS, false>();
#else
  (void)mask;
  return KernelInfo{nullptr, 0, 0, 0, 0};
#endif
}

}  // namespace lbf
