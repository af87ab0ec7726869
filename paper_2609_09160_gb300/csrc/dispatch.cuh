// Launch-time dispatch from runtime parameters (lattice, storage dtype, mask, two-component) to the
// kernel template instantiations. Each lattice's kernels are instantiated in their own
// translation unit (kernels_d3q19.cu, kernels_d3q27.cu) so they compile in parallel.
#pragma once

#include "adjoint.cuh"
#include "stream_collide.cuh"

namespace lbf {

enum StorageId { ST_F64 = 0, ST_F32 = 1, ST_F16 = 2, ST_BF16 = 3 };

// tile rows (output rows per CTA) by compute precision: FP64 rings are twice as large
constexpr int tile_rows(int storage) { return storage == ST_F64 ? 4 : 8; }

struct KernelInfo {
  const void* fn;   // kernel entry point
  size_t smem;      // dynamic shared memory bytes
  int threads;      // threads per CTA
  int by;           // output rows per CTA
};

template <class L, class S, bool MASK, bool TWO>
KernelInfo fwd_info() {
  using T = typename ComputeOf<S>::type;
  constexpr int BY = std::is_same<S, double>::value ? 4 : 8;
  KernelInfo k;
  k.fn = reinterpret_cast<const void*>(&k_stream_collide<L, S, BY, MASK, TWO>);
  k.smem = fwd_smem_bytes<L, T, BY, MASK>();
  k.threads = FwdTile<BY>::THREADS;
  k.by = BY;
  return k;
}

template <class L, class S, bool MASK>
KernelInfo adj_info() {
  using T = typename ComputeOf<S>::type;
  constexpr int BY = std::is_same<S, double>::value ? 4 : 8;
  KernelInfo k;
  k.fn = reinterpret_cast<const void*>(&k_adjoint<L, S, BY, MASK>);
  k.smem = fwd_smem_bytes<L, T, BY, MASK>();
  k.threads = FwdTile<BY>::THREADS;
  k.by = BY;
  return k;
}

// forward kernel for (storage, mask, two) of lattice L; fn == nullptr if not built
template <class L>
KernelInfo forward_kernel(int storage, bool mask, bool two) {
  if (mask && two) return KernelInfo{nullptr, 0, 0, 0};
  switch (storage) {
    case ST_F64:
      return mask ? fwd_info<L, double, true, false>() : (two ? fwd_info<L, double, false, true>() : fwd_info<L, double, false, false>());
    case ST_F32:
      return mask ? fwd_info<L, float, true, false>() : (two ? fwd_info<L, float, false, true>() : fwd_info<L, float, false, false>());
    case ST_F16:
      return mask ? fwd_info<L, __half, true, false>() : (two ? fwd_info<L, __half, false, true>() : fwd_info<L, __half, false, false>());
    case ST_BF16:
      return mask ? fwd_info<L, __nv_bfloat16, true, false>()
                  : (two ? fwd_info<L, __nv_bfloat16, false, true>() : fwd_info<L, __nv_bfloat16, false, false>());
  }
  return KernelInfo{nullptr, 0, 0, 0};
}

template <class L>
KernelInfo adjoint_kernel(int storage, bool mask) {
  switch (storage) {
    case ST_F64:
      return mask ? adj_info<L, double, true>() : adj_info<L, double, false>();
    case ST_F32:
      return mask ? adj_info<L, float, true>() : adj_info<L, float, false>();
  }
  return KernelInfo{nullptr, 0, 0, 0};
}

// entry points implemented per lattice (one translation unit each)
KernelInfo forward_kernel_q19(int storage, bool mask, bool two);
KernelInfo forward_kernel_q27(int storage, bool mask, bool two);
KernelInfo adjoint_kernel_q19(int storage, bool mask);
KernelInfo adjoint_kernel_q27(int storage, bool mask);

}  // namespace lbf
