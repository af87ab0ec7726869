// Compile-time D3Q19 / D3Q27 velocity sets and small device helpers for the fused kernels.
//
// The paper states the method for any quadrature (Sec. 2, "Eq. (pullLLB) is formulated in a way
// that is independent of the specific choice of the discrete velocity set") and uses D3Q19 and
// D3Q27 with the Hermite expansion truncated at second order. Directions are numbered from the
// 3x3x3 cube, q27 = 9 (cz+1) + 3 (cy+1) + (cx+1), so the opposite of q27 is 26 - q27. D3Q19 keeps
// the 19 entries with |c|^2 <= 2 in the same order, so its opposite is 18 - q.
// Weights: D3Q19 1/3, 1/18, 1/36; D3Q27 8/27, 2/27, 1/54, 1/216 by |c|^2 (c_s^2 = 1/3).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <utility>

namespace lbf {

struct D3Q27 {
  static constexpr int Q = 27;
  __host__ __device__ static constexpr int cube(int q) { return q; }
  __host__ __device__ static constexpr int cx(int q) { return cube(q) % 3 - 1; }
  __host__ __device__ static constexpr int cy(int q) { return (cube(q) / 3) % 3 - 1; }
  __host__ __device__ static constexpr int cz(int q) { return cube(q) / 9 - 1; }
  __host__ __device__ static constexpr int opp(int q) { return Q - 1 - q; }
  __host__ __device__ static constexpr double w(int q) {
    return (cx(q) * cx(q) + cy(q) * cy(q) + cz(q) * cz(q)) == 0   ? 8.0 / 27.0
           : (cx(q) * cx(q) + cy(q) * cy(q) + cz(q) * cz(q)) == 1 ? 2.0 / 27.0
           : (cx(q) * cx(q) + cy(q) * cy(q) + cz(q) * cz(q)) == 2 ? 1.0 / 54.0
                                                                   : 1.0 / 216.0;
  }
  static constexpr bool HIGH = false;  // second-order Hermite truncation
  static constexpr const char* name = "D3Q27";
};

// D3Q27h (Sec. 2): the D3Q27 velocities with the complete Hermite basis; the post-collision
// populations carry every Hermite coefficient the lattice supports, the higher ones reconstructed
// from p*, u, N and F by the recursive closure
struct D3Q27H : D3Q27 {
  static constexpr bool HIGH = true;
  static constexpr const char* name = "D3Q27H";
};

struct D3Q19 {
  static constexpr int Q = 19;
  // q-th cube index whose |c|^2 <= 2 (the 8 corners are skipped)
  __host__ __device__ static constexpr int cube(int q) {
    int seen = -1;
    for (int k = 0; k < 27; ++k) {
      const int x = k % 3 - 1, y = (k / 3) % 3 - 1, z = k / 9 - 1;
      if (x * x + y * y + z * z <= 2) {
        ++seen;
        if (seen == q) return k;
      }
    }
    return -1;
  }
  __host__ __device__ static constexpr int cx(int q) { return cube(q) % 3 - 1; }
  __host__ __device__ static constexpr int cy(int q) { return (cube(q) / 3) % 3 - 1; }
  __host__ __device__ static constexpr int cz(int q) { return cube(q) / 9 - 1; }
  __host__ __device__ static constexpr int opp(int q) { return Q - 1 - q; }
  __host__ __device__ static constexpr double w(int q) {
    return (cx(q) * cx(q) + cy(q) * cy(q) + cz(q) * cz(q)) == 0   ? 1.0 / 3.0
           : (cx(q) * cx(q) + cy(q) * cy(q) + cz(q) * cz(q)) == 1 ? 1.0 / 18.0
                                                                   : 1.0 / 36.0;
  }
  static constexpr bool HIGH = false;
  static constexpr const char* name = "D3Q19";
};

template <class L>
__host__ __device__ constexpr int rest_index() {
  for (int q = 0; q < L::Q; ++q)
    if (L::cx(q) == 0 && L::cy(q) == 0 && L::cz(q) == 0) return q;
  return -1;
}

// compile-time loop: f(std::integral_constant<int, I>{}) for I = 0 .. N-1
template <class F, int... I>
__device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// ---------------------------------------------------------------------------------------------
// Storage codec. The state keeps 10 fields per site: p*, u (3) and the non-equilibrium part of
// the second Hermite coefficient, N = a2 - u u (6), each group g in {p, u, N} multiplied by a
// power-of-two scale 2^s_g before it is rounded to the storage type (round to nearest even).
// For FP32 and FP64 the scales are 1 and the multiply is compiled out.
template <class S>
struct Codec;

// store: round to nearest (loading a state; the N fields of a step). store_sr: unbiased
// stochastic rounding with the random word r, used by the time step for p* and u. Round-to-nearest
// of a 16-bit state discards every update smaller than half a unit in the last place: on large
// lattices, where the flow changes by less than 2^-12 of its value per step, the state then
// freezes and its error grows with time.
// Adding uniform random bits below the kept significand and truncating rounds up with
// probability equal to the discarded fraction, so the expected stored value is exact.
template <>
struct Codec<double> {
  static constexpr bool scaled = false;
  __device__ __forceinline__ static double load(const double* p) { return __ldg(p); }
  __device__ __forceinline__ static void store(double* p, double v) { *p = v; }
  __device__ __forceinline__ static void store_sr(double* p, double v, uint32_t) { *p = v; }
};
template <>
struct Codec<float> {
  static constexpr bool scaled = false;
  __device__ __forceinline__ static float load(const float* p) { return __ldg(p); }
  __device__ __forceinline__ static void store(float* p, float v) { *p = v; }
  __device__ __forceinline__ static void store_sr(float* p, float v, uint32_t) { *p = v; }
};
template <>
struct Codec<__half> {
  static constexpr bool scaled = true;
  __device__ __forceinline__ static float load(const __half* p) { return __half2float(__ldg(p)); }
  __device__ __forceinline__ static void store(__half* p, float v) { *p = __float2half_rn(v); }
  // FP16 keeps 10 of FP32's 23 significand bits: 13 random bits, then round toward zero
  __device__ __forceinline__ static void store_sr(__half* p, float v, uint32_t r) {
    *p = __float2half_rz(__uint_as_float(__float_as_uint(v) + (r >> 19)));
  }
};
template <>
struct Codec<__nv_bfloat16> {
  static constexpr bool scaled = true;
  __device__ __forceinline__ static float load(const __nv_bfloat16* p) {
    return __bfloat162float(__ldg(p));
  }
  __device__ __forceinline__ static void store(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
  // BF16 is the upper half of FP32: 16 random bits, then truncation
  __device__ __forceinline__ static void store_sr(__nv_bfloat16* p, float v, uint32_t r) {
    *p = __ushort_as_bfloat16(static_cast<unsigned short>((__float_as_uint(v) + (r >> 16)) >> 16));
  }
};

// Counter-based random words for stochastic rounding. fmix32 is the 32-bit finaliser of
// MurmurHash3 (A. Appleby): a bijective mixer that turns a counter into a uniformly distributed
// word. Successive words for one site come from the linear congruential step of the PCG family
// (M. E. O'Neill: multiplier 747796405, increment 2891336453); the high bits are used.
__host__ __device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}
__device__ __forceinline__ uint32_t lcg_next(uint32_t s) { return s * 747796405u + 2891336453u; }

// per-group scale factors passed by value to every kernel
struct Scales {
  float enc[3];  // p, u, N: stored = value * enc
  float dec[3];  // value = stored * dec
};

// signed add of a compile-time coefficient in {-1, 0, 1}: no arithmetic when it is 0
template <int C, class T>
__device__ __forceinline__ T sadd(T acc, T v) {
  if constexpr (C > 0)
    return acc + v;
  else if constexpr (C < 0)
    return acc - v;
  else
    return acc;
}

__device__ __forceinline__ int wrap(int i, int n) {
  // i in [-n, 2n): periodic index
  return i < 0 ? i + n : (i >= n ? i - n : i);
}

}  // namespace lbf
