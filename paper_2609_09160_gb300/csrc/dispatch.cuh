// Launch-time dispatch from runtime parameters (lattice, storage dtype, mask, two-component) to the
// kernel template instantiations. Each lattice's kernels are instantiated in their own
// translation unit (kernels_d3q19.cu, kernels_d3q27.cu) so they compile in parallel.
#pragma once

#include "adjoint.cuh"
#include "stream_collide.cuh"

namespace lbf {

enum StorageId { ST_F64 = 0, ST_F32 = 1, ST_F16 = 2, ST_BF16 = 3 };

// output rows per CTA of the forward kernel (FP32 compute / FP64 compute) and of the adjoint
#ifndef LBF_FWD_ROWS
#define LBF_FWD_ROWS 8
#endif
#ifndef LBF_FWD_ROWS_F64
#define LBF_FWD_ROWS_F64 4
#endif
constexpr int fwd_rows(bool fp64) { return fp64 ? LBF_FWD_ROWS_F64 : LBF_FWD_ROWS; }
constexpr int adj_rows(bool fp64) { return fp64 ? 4 : 8; }

struct KernelInfo {
  const void* fn;   // kernel entry point
  size_t smem;      // dynamic shared memory bytes
  int threads;      // threads per CTA
  int by;           // output rows per CTA
  int box_x;        // TMA box width in elements (0: the kernel loads without TMA)
};

template <class L, class S, bool MASK, bool TWO, bool TMA>
KernelInfo fwd_info() {
  constexpr int BY = fwd_rows(std::is_same<S, double>::value);
  KernelInfo k;
  k.fn = reinterpret_cast<const void*>(&k_stream_collide<L, S, BY, MASK, TWO, TMA>);
  k.smem = fwd_smem_bytes<L, S, BY, MASK, TMA>();
  k.threads = FwdTile<BY>::THREADS;
  k.by = BY;
  k.box_x = TMA ? TmaBox<S>::BX : 0;
  return k;
}

template <class L, class S, bool MASK>
KernelInfo adj_info() {
  using T = typename ComputeOf<S>::type;
  constexpr int BY = adj_rows(std::is_same<S, double>::value);
  KernelInfo k;
  k.fn = reinterpret_cast<const void*>(&k_adjoint<L, S, BY, MASK>);
  k.smem = ring3_smem_bytes<L, T, BY, MASK>();
  k.threads = FwdTile<BY>::THREADS;
  k.by = BY;
  k.box_x = 0;
  return k;
}

template <class L, class S, bool TMA>
KernelInfo forward_kernel_s(bool mask, bool two) {
  if (mask) return fwd_info<L, S, true, false, TMA>();
  return two ? fwd_info<L, S, false, true, TMA>() : fwd_info<L, S, false, false, TMA>();
}

// forward kernel for (storage, mask, two, tma) of lattice L; fn == nullptr if not built
template <class L>
KernelInfo forward_kernel(int storage, bool mask, bool two, bool tma) {
  if (mask && two) return KernelInfo{nullptr, 0, 0, 0, 0};
  switch (storage) {
    case ST_F64: return tma ? forward_kernel_s<L, double, true>(mask, two) : forward_kernel_s<L, double, false>(mask, two);
    case ST_F32: return tma ? forward_kernel_s<L, float, true>(mask, two) : forward_kernel_s<L, float, false>(mask, two);
    case ST_F16: return tma ? forward_kernel_s<L, __half, true>(mask, two) : forward_kernel_s<L, __half, false>(mask, two);
    case ST_BF16:
      return tma ? forward_kernel_s<L, __nv_bfloat16, true>(mask, two) : forward_kernel_s<L, __nv_bfloat16, false>(mask, two);
  }
  return KernelInfo{nullptr, 0, 0, 0, 0};
}

template <class L>
KernelInfo adjoint_kernel(int storage, bool mask) {
  switch (storage) {
    case ST_F64:
      return mask ? adj_info<L, double, true>() : adj_info<L, double, false>();
    case ST_F32:
      return mask ? adj_info<L, float, true>() : adj_info<L, float, false>();
  }
  return KernelInfo{nullptr, 0, 0, 0, 0};
}

// entry points implemented per lattice (one translation unit each)
KernelInfo forward_kernel_q19(int storage, bool mask, bool two, bool tma);
KernelInfo forward_kernel_q27(int storage, bool mask, bool two, bool tma);
KernelInfo adjoint_kernel_q19(int storage, bool mask);
KernelInfo adjoint_kernel_q27(int storage, bool mask);

}  // namespace lbf
