// Helper kernels around the fused step: state encode/decode (public layout <-> storage), the
// 16-bit scale search, the standalone and final conservation reductions, and the two-component
// phase-field update (Eq. ACeq) with the capillary force.
#pragma once

#include "lattice.cuh"

namespace lbf {

// public [10][stride] (site i of the chunk) -> internal state at site0 + i
template <class Tin, class S>
__global__ void k_encode(const Tin* __restrict__ src, long long stride, long long site0, long long count,
                         S* __restrict__ dst, long long N, Scales sc) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    double v[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) v[k] = static_cast<double>(src[k * stride + i]);
    const double ux = v[1], uy = v[2], uz = v[3];
    double n[6] = {v[4] - ux * ux, v[5] - uy * uy, v[6] - uz * uz,
                   v[7] - ux * uy, v[8] - ux * uz, v[9] - uy * uz};
    const long long s = site0 + i;
    if constexpr (Codec<S>::scaled) {
      Codec<S>::store(dst + s, static_cast<float>(v[0] * sc.enc[0]));
      for (int k = 1; k < 4; ++k) Codec<S>::store(dst + k * N + s, static_cast<float>(v[k] * sc.enc[1]));
      for (int k = 0; k < 6; ++k) Codec<S>::store(dst + (4 + k) * N + s, static_cast<float>(n[k] * sc.enc[2]));
    } else {
      dst[s] = static_cast<S>(v[0]);
      for (int k = 1; k < 4; ++k) dst[k * N + s] = static_cast<S>(v[k]);
      for (int k = 0; k < 6; ++k) dst[(4 + k) * N + s] = static_cast<S>(n[k]);
    }
  }
}

// internal state at site0 + i -> public [10][stride]
template <class S, class Tout>
__global__ void k_decode(const S* __restrict__ src, long long N, long long site0, long long count,
                         Tout* __restrict__ dst, long long stride, Scales sc) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const long long s = site0 + i;
    double v[10];
    if constexpr (Codec<S>::scaled) {
      v[0] = static_cast<double>(Codec<S>::load(src + s)) * sc.dec[0];
      for (int k = 1; k < 4; ++k) v[k] = static_cast<double>(Codec<S>::load(src + k * N + s)) * sc.dec[1];
      for (int k = 4; k < 10; ++k) v[k] = static_cast<double>(Codec<S>::load(src + k * N + s)) * sc.dec[2];
    } else {
      for (int k = 0; k < 10; ++k) v[k] = static_cast<double>(src[k * N + s]);
    }
    const double ux = v[1], uy = v[2], uz = v[3];
    v[4] += ux * ux;
    v[5] += uy * uy;
    v[6] += uz * uz;
    v[7] += ux * uy;
    v[8] += ux * uz;
    v[9] += uy * uz;
#pragma unroll
    for (int k = 0; k < 10; ++k) dst[k * stride + i] = static_cast<Tout>(v[k]);
  }
}

// max |p*|, |u|, |A - u u| of a public chunk, as float bit patterns (non-negative floats order
// like their bits), into out[0..2] (atomicMax)
template <class Tin>
__global__ void k_absmax(const Tin* __restrict__ src, long long stride, long long count, unsigned* out) {
  float m[3] = {0.f, 0.f, 0.f};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    double v[10];
    for (int k = 0; k < 10; ++k) v[k] = static_cast<double>(src[k * stride + i]);
    const double ux = v[1], uy = v[2], uz = v[3];
    m[0] = fmaxf(m[0], (float)fabs(v[0]));
    m[1] = fmaxf(m[1], (float)fmax(fabs(ux), fmax(fabs(uy), fabs(uz))));
    const double n[6] = {v[4] - ux * ux, v[5] - uy * uy, v[6] - uz * uz, v[7] - ux * uy, v[8] - ux * uz, v[9] - uy * uz};
    for (int k = 0; k < 6; ++k) m[2] = fmaxf(m[2], (float)fabs(n[k]));
  }
  for (int k = 0; k < 3; ++k) {
    float x = m[k];
    for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out + k, __float_as_uint(x));
  }
}

// conservation sums of a state over fluid sites, one FP64 partial (8 doubles) per block
template <class S>
__global__ void k_reduce_state(const S* __restrict__ st, long long N, const uint8_t* __restrict__ mask,
                               const void* phi, bool phi_double, Scales sc, double* partials) {
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N;
       s += (long long)gridDim.x * blockDim.x) {
    if (mask != nullptr && mask[s]) continue;
    double v[4];
    if constexpr (Codec<S>::scaled) {
      v[0] = static_cast<double>(Codec<S>::load(st + s)) * sc.dec[0];
      for (int k = 1; k < 4; ++k) v[k] = static_cast<double>(Codec<S>::load(st + k * N + s)) * sc.dec[1];
    } else {
      for (int k = 0; k < 4; ++k) v[k] = static_cast<double>(st[k * N + s]);
    }
    acc[0] += v[0];
    acc[1] += v[1];
    acc[2] += v[2];
    acc[3] += v[3];
    if (phi != nullptr)
      acc[4] += phi_double ? static_cast<const double*>(phi)[s] : static_cast<double>(static_cast<const float*>(phi)[s]);
    acc[5] += v[1] * v[1] + v[2] * v[2] + v[3] * v[3];
  }
  __shared__ double sh[32][6];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int k = 0; k < 6; ++k) {
    double x = acc[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) sh[wid][k] = x;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w][threadIdx.x];
    partials[blockIdx.x * 8 + threadIdx.x] = s;
  }
}

// deterministic sum of nblocks partials (one block of 256 threads, fixed order)
__global__ void k_reduce_final(const double* __restrict__ partials, long long nblocks, double* out) {
  __shared__ double sh[256][6];
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (long long b = threadIdx.x; b < nblocks; b += blockDim.x)
    for (int k = 0; k < 6; ++k) acc[k] += partials[b * 8 + k];
  for (int k = 0; k < 6; ++k) sh[threadIdx.x][k] = acc[k];
  __syncthreads();
  for (int step = 128; step > 0; step >>= 1) {
    if ((int)threadIdx.x < step)
      for (int k = 0; k < 6; ++k) sh[threadIdx.x][k] += sh[threadIdx.x + step][k];
    __syncthreads();
  }
  if (threadIdx.x < 6) out[threadIdx.x] = sh[0][threadIdx.x];
}

// ---------------------------------------------------------------------------------------------
// Two-component coupling (Sec. 2): D3Q27-weight stencils,
//   grad psi = 3 sum_i w_i c_i psi(x + c_i),  lap psi = 6 sum_i w_i (psi(x + c_i) - psi(x)),
//   div V = 3 sum_i w_i c_i . V(x + c_i)
// Allen-Cahn FTCS in flux form: phi' = phi - div(phi u) + D lap phi - lambda div(G),
// G = phi (1 - phi) n, n = grad phi / max(|grad phi|, 1e-12), lambda = 4 D / W.
struct PhaseParams {
  int nx, ny, nz;
  long long N;
  double D, lambda, beta, kappa;
  double body[3];
  Scales sc;
};

__device__ __forceinline__ long long site_of(int x, int y, int z, int nx, int ny) {
  return ((long long)z * ny + y) * nx + x;
}

// phi_new from phi, u (decoded from the state) and G, all at time n
template <class S, class T>
__global__ void k_phase_advance(const S* __restrict__ st, const T* __restrict__ phi, const T* __restrict__ G,
                                T* __restrict__ phi_new, PhaseParams p) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z * blockDim.z + threadIdx.z;
  if (x >= p.nx || y >= p.ny || z >= p.nz) return;
  const long long N = p.N;
  const long long s0 = site_of(x, y, z, p.nx, p.ny);
  const T ph0 = phi[s0];
  T div_adv = T(0), lap = T(0), div_g = T(0);
  static_for<27>([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    constexpr int cx = D3Q27::cx(q), cy = D3Q27::cy(q), cz = D3Q27::cz(q);
    if constexpr (cx != 0 || cy != 0 || cz != 0) {
      constexpr T w = T(D3Q27::w(q));
      const int xs = wrap(x + cx, p.nx), ys = wrap(y + cy, p.ny), zs = wrap(z + cz, p.nz);
      const long long s = site_of(xs, ys, zs, p.nx, p.ny);
      const T ph = phi[s];
      lap += w * (ph - ph0);
      T ux, uy, uz;
      if constexpr (Codec<S>::scaled) {
        ux = Codec<S>::load(st + N + s) * p.sc.dec[1];
        uy = Codec<S>::load(st + 2 * N + s) * p.sc.dec[1];
        uz = Codec<S>::load(st + 3 * N + s) * p.sc.dec[1];
      } else {
        ux = st[N + s];
        uy = st[2 * N + s];
        uz = st[3 * N + s];
      }
      T cu = T(0), cg = T(0);
      if constexpr (cx != 0) {
        cu = sadd<cx>(cu, ph * ux);
        cg = sadd<cx>(cg, G[s]);
      }
      if constexpr (cy != 0) {
        cu = sadd<cy>(cu, ph * uy);
        cg = sadd<cy>(cg, G[N + s]);
      }
      if constexpr (cz != 0) {
        cu = sadd<cz>(cu, ph * uz);
        cg = sadd<cz>(cg, G[2 * N + s]);
      }
      div_adv += w * cu;
      div_g += w * cg;
    }
  });
  phi_new[s0] = ph0 - T(3) * div_adv + T(p.D) * T(6) * lap - T(p.lambda) * T(3) * div_g;
}

// force F = mu grad phi + F^b and compression flux G from phi (time n+1)
template <class T>
__global__ void k_phase_forces(const T* __restrict__ phi, T* __restrict__ F, T* __restrict__ G, PhaseParams p) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z * blockDim.z + threadIdx.z;
  if (x >= p.nx || y >= p.ny || z >= p.nz) return;
  const long long N = p.N;
  const long long s0 = site_of(x, y, z, p.nx, p.ny);
  const T ph0 = phi[s0];
  T gx = T(0), gy = T(0), gz = T(0), lap = T(0);
  static_for<27>([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    constexpr int cx = D3Q27::cx(q), cy = D3Q27::cy(q), cz = D3Q27::cz(q);
    if constexpr (cx != 0 || cy != 0 || cz != 0) {
      constexpr T w = T(D3Q27::w(q));
      const int xs = wrap(x + cx, p.nx), ys = wrap(y + cy, p.ny), zs = wrap(z + cz, p.nz);
      const T ph = phi[site_of(xs, ys, zs, p.nx, p.ny)];
      lap += w * (ph - ph0);
      if constexpr (cx != 0) gx = sadd<cx>(gx, w * ph);
      if constexpr (cy != 0) gy = sadd<cy>(gy, w * ph);
      if constexpr (cz != 0) gz = sadd<cz>(gz, w * ph);
    }
  });
  gx *= T(3);
  gy *= T(3);
  gz *= T(3);
  lap *= T(6);
  const T mu = T(4) * T(p.beta) * ph0 * (ph0 - T(1)) * (ph0 - T(0.5)) - T(p.kappa) * lap;
  F[s0] = mu * gx + T(p.body[0]);
  F[N + s0] = mu * gy + T(p.body[1]);
  F[2 * N + s0] = mu * gz + T(p.body[2]);
  T mag = sqrt(gx * gx + gy * gy + gz * gz);
  mag = mag > T(1e-12) ? mag : T(1e-12);
  const T c = ph0 * (T(1) - ph0) / mag;
  G[s0] = c * gx;
  G[N + s0] = c * gy;
  G[2 * N + s0] = c * gz;
}

}  // namespace lbf
