// Launch-time dispatch from runtime parameters (lattice, storage dtype, mask, force mode) to the
// kernel template instantiations. The kernels of each (lattice, storage) pair are instantiated in
// their own translation unit (kernels.cu compiled once per pair) so they compile in parallel.
#pragma once

#include "adjoint.cuh"
#include "population.cuh"
#include "stream_collide.cuh"
#include "stream_collide_aligned.cuh"

namespace lbf {

enum StorageId { ST_F64 = 0, ST_F32 = 1, ST_F16 = 2, ST_BF16 = 3 };

// output rows per CTA of the adjoint kernel (FP32 compute / FP64 compute); the forward kernel's
// are fwd_rows() of stream_collide.cuh
constexpr int adj_rows(bool fp64) { return fp64 ? 4 : 8; }

struct KernelInfo {
  const void* fn;   // kernel entry point
  size_t smem;      // dynamic shared memory bytes
  int threads;      // threads per CTA
  int by;           // output rows per CTA
  int box_x;        // TMA box width in elements (0: the kernel loads without TMA)
  int xout = 30;    // output columns per CTA: 30 (k_stream_collide) or 32 (k_stream_collide_al)
  bool store_map = false;  // the kernel also takes a tensor map of dst (TMA stores)
};

template <class L, class S, bool MASK, int TWO, bool FF, bool TMA, bool RN>
KernelInfo fwd_info() {
  constexpr int BY = fwd_rows_lattice(L::Q, int(sizeof(S)), MASK, TWO != 0, L::HIGH);
  KernelInfo k;
  k.fn = reinterpret_cast<const void*>(&k_stream_collide<L, S, BY, MASK, TWO, FF, TMA, RN>);
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

// forward kernel of lattice L and storage S for (mask, two-component mode, force field, TMA,
// 16-bit round-to-nearest); two: 0 single component, 1 two components at equal densities, 2 with a
// density contrast. fn == nullptr for combinations that are not built (two components with a force
// field; a contrast or walls with two components in 16-bit storage). Round-to-nearest kernels exist
// for 16-bit storage only (FP32/FP64 stores are exact).
template <class L, class S, bool TMA, bool RN>
KernelInfo forward_kernel_s(bool mask, int two, bool field) {
  constexpr bool wide = !Codec<S>::scaled;  // FP32 / FP64 storage
  if (two != 0 && field) return KernelInfo{nullptr, 0, 0, 0, 0};
  if (two == 2) {
    if constexpr (wide)
      return mask ? fwd_info<L, S, true, 2, false, TMA, RN>() : fwd_info<L, S, false, 2, false, TMA, RN>();
    else
      return KernelInfo{nullptr, 0, 0, 0, 0};
  }
  if (two == 1) {
    if (!mask) return fwd_info<L, S, false, 1, false, TMA, RN>();
    if constexpr (wide)
      return fwd_info<L, S, true, 1, false, TMA, RN>();
    else
      return KernelInfo{nullptr, 0, 0, 0, 0};
  }
  if (mask) return field ? fwd_info<L, S, true, 0, true, TMA, RN>() : fwd_info<L, S, true, 0, false, TMA, RN>();
  return field ? fwd_info<L, S, false, 0, true, TMA, RN>() : fwd_info<L, S, false, 0, false, TMA, RN>();
}

template <class L, class S>
KernelInfo forward_kernel_ls(bool mask, int two, bool field, bool tma, bool nearest) {
  if constexpr (Codec<S>::scaled) {
    if (nearest)
      return tma ? forward_kernel_s<L, S, true, true>(mask, two, field)
                 : forward_kernel_s<L, S, false, true>(mask, two, field);
  }
  return tma ? forward_kernel_s<L, S, true, false>(mask, two, field)
             : forward_kernel_s<L, S, false, false>(mask, two, field);
}

// line-aligned kernel with TMA stores (FP32 and 16-bit storage, single component)
template <class L, class S, bool MASK, bool FF, bool RN>
KernelInfo al_info() {
  constexpr int TY = al_rows(L::Q, int(sizeof(S)), MASK, L::HIGH);
  KernelInfo k;
  k.fn = reinterpret_cast<const void*>(&k_stream_collide_al<L, S, TY, MASK, FF, RN>);
  k.smem = al_smem_bytes<L, S, TY, MASK>();
  k.threads = AlTile<S, TY>::THREADS;
  k.by = TY;
  k.box_x = AlTile<S, TY>::BX;
  k.xout = 32;
  k.store_map = true;
  return k;
}

template <class L, class S, bool RN>
KernelInfo aligned_kernel_s(bool mask, bool field) {
  if (mask) return field ? al_info<L, S, true, true, RN>() : al_info<L, S, true, false, RN>();
  return field ? al_info<L, S, false, true, RN>() : al_info<L, S, false, false, RN>();
}

template <class L, class S>
KernelInfo aligned_kernel_ls(bool mask, bool field, bool nearest) {
  if constexpr (std::is_same<S, double>::value) {
    (void)mask;
    (void)field;
    (void)nearest;
    return KernelInfo{nullptr, 0, 0, 0, 0};  // FP64 storage keeps the 30-column kernel
  } else {
    if constexpr (Codec<S>::scaled) {
      if (nearest) return aligned_kernel_s<L, S, true>(mask, field);
    }
    return aligned_kernel_s<L, S, false>(mask, field);
  }
}

// population-form reference kernels of lattice L, storage S (FP32/FP64 only; nulls otherwise)
struct PopKernels {
  const void* step;     // k_pop_step
  const void* init;     // k_pop_from_moments
  const void* moments;  // k_pop_moments
};

template <class L, class T, bool MASK, bool FF>
PopKernels pop_kernels_info() {
  return PopKernels{reinterpret_cast<const void*>(&k_pop_step<L, T, MASK, FF>),
                    reinterpret_cast<const void*>(&k_pop_from_moments<L, T, FF>),
                    reinterpret_cast<const void*>(&k_pop_moments<L, T, MASK, FF>)};
}

template <class L, class S>
PopKernels pop_kernels_ls(bool mask, bool field) {
  if constexpr (std::is_same<S, float>::value || std::is_same<S, double>::value) {
    if (mask) return field ? pop_kernels_info<L, S, true, true>() : pop_kernels_info<L, S, true, false>();
    return field ? pop_kernels_info<L, S, false, true>() : pop_kernels_info<L, S, false, false>();
  } else {
    (void)mask;
    (void)field;
    return PopKernels{nullptr, nullptr, nullptr};
  }
}

// entry points implemented per (lattice, storage) translation unit
#define LBF_DECLARE_TU(q, s)                                                             \
  KernelInfo forward_kernel_q##q##_s##s(bool mask, int two, bool field, bool tma, bool nearest); \
  KernelInfo aligned_kernel_q##q##_s##s(bool mask, bool field, bool nearest);                    \
  PopKernels pop_kernels_q##q##_s##s(bool mask, bool field);                                        \
  KernelInfo adjoint_kernel_q##q##_s##s(bool mask);
LBF_DECLARE_TU(19, 0)
LBF_DECLARE_TU(19, 1)
LBF_DECLARE_TU(19, 2)
LBF_DECLARE_TU(19, 3)
LBF_DECLARE_TU(27, 0)
LBF_DECLARE_TU(27, 1)
LBF_DECLARE_TU(27, 2)
LBF_DECLARE_TU(27, 3)
LBF_DECLARE_TU(127, 0)
LBF_DECLARE_TU(127, 1)
LBF_DECLARE_TU(127, 2)
LBF_DECLARE_TU(127, 3)
#undef LBF_DECLARE_TU

// lattice: 19 (D3Q19), 27 (D3Q27) or 127 (D3Q27h: D3Q27 with the complete Hermite basis)
inline KernelInfo forward_kernel_for(int lattice, int storage, bool mask, int two, bool field, bool tma,
                                     bool nearest) {
  const bool q19 = lattice == 19;
  if (lattice == 127) {
    switch (storage) {
      case ST_F64: return forward_kernel_q127_s0(mask, two, field, tma, nearest);
      case ST_F32: return forward_kernel_q127_s1(mask, two, field, tma, nearest);
      case ST_F16: return forward_kernel_q127_s2(mask, two, field, tma, nearest);
      case ST_BF16: return forward_kernel_q127_s3(mask, two, field, tma, nearest);
    }
    return KernelInfo{nullptr, 0, 0, 0, 0};
  }
  switch (storage) {
    case ST_F64:
      return q19 ? forward_kernel_q19_s0(mask, two, field, tma, nearest) : forward_kernel_q27_s0(mask, two, field, tma, nearest);
    case ST_F32:
      return q19 ? forward_kernel_q19_s1(mask, two, field, tma, nearest) : forward_kernel_q27_s1(mask, two, field, tma, nearest);
    case ST_F16:
      return q19 ? forward_kernel_q19_s2(mask, two, field, tma, nearest) : forward_kernel_q27_s2(mask, two, field, tma, nearest);
    case ST_BF16:
      return q19 ? forward_kernel_q19_s3(mask, two, field, tma, nearest) : forward_kernel_q27_s3(mask, two, field, tma, nearest);
  }
  return KernelInfo{nullptr, 0, 0, 0, 0};
}

// line-aligned kernel with TMA stores; fn == nullptr where it is not built (FP64 storage)
inline KernelInfo aligned_kernel_for(int lattice, int storage, bool mask, bool field, bool nearest) {
#define LBF_AL_CASE(q)                                                     \
  switch (storage) {                                                      \
    case ST_F64: return aligned_kernel_q##q##_s0(mask, field, nearest);   \
    case ST_F32: return aligned_kernel_q##q##_s1(mask, field, nearest);   \
    case ST_F16: return aligned_kernel_q##q##_s2(mask, field, nearest);   \
    case ST_BF16: return aligned_kernel_q##q##_s3(mask, field, nearest);  \
  }
  if (lattice == 19) {
    LBF_AL_CASE(19)
  } else if (lattice == 27) {
    LBF_AL_CASE(27)
  } else if (lattice == 127) {
    LBF_AL_CASE(127)
  }
#undef LBF_AL_CASE
  return KernelInfo{nullptr, 0, 0, 0, 0};
}

inline PopKernels pop_kernels_for(int lattice, int storage, bool mask, bool field) {
  if (lattice == 127) return PopKernels{nullptr, nullptr, nullptr};  // second-order collision only
  const bool q19 = lattice == 19;
  switch (storage) {
    case ST_F64: return q19 ? pop_kernels_q19_s0(mask, field) : pop_kernels_q27_s0(mask, field);
    case ST_F32: return q19 ? pop_kernels_q19_s1(mask, field) : pop_kernels_q27_s1(mask, field);
  }
  return PopKernels{nullptr, nullptr, nullptr};
}

// adjoint kernel (FP64 and FP32 storage only; fn == nullptr otherwise)
inline KernelInfo adjoint_kernel_for(int lattice, int storage, bool mask) {
  if (lattice == 127) return KernelInfo{nullptr, 0, 0, 0, 0};  // the adjoint is of the second-order step
  const bool q19 = lattice == 19;
  switch (storage) {
    case ST_F64: return q19 ? adjoint_kernel_q19_s0(mask) : adjoint_kernel_q27_s0(mask);
    case ST_F32: return q19 ? adjoint_kernel_q19_s1(mask) : adjoint_kernel_q27_s1(mask);
    case ST_F16: return q19 ? adjoint_kernel_q19_s2(mask) : adjoint_kernel_q27_s2(mask);
    case ST_BF16: return q19 ? adjoint_kernel_q19_s3(mask) : adjoint_kernel_q27_s3(mask);
  }
  return KernelInfo{nullptr, 0, 0, 0, 0};
}

}  // namespace lbf
