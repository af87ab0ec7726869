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
//
// The D3Q27 weights are products of one-dimensional weights, w_i = a(c_x) a(c_y) a(c_z) with
// a(0) = 2/3 and a(+-1) = 1/6, so every stencil above separates into three-point filters along
// the axes: the smoothing A f = a(0) f(0) + a(1) (f(-1) + f(+1)) and the difference
// D f = (f(+1) - f(-1)) / 6, e.g. sum_i w_i c_i,x psi(x + c_i) = D_x A_y A_z psi and
// sum_i w_i psi(x + c_i) = A_x A_y A_z psi. The Laplacian is assembled from second differences
// only, with L = A - I = (1/6) [1, -2, 1]:
//   sum_i w_i (psi(x + c_i) - psi(x)) = L_x A_y psi + L_y psi + A_x A_y L_z psi,
// so that, as in the flux form, every term vanishes exactly on a constant field: the rounded
// weights 2/3 and 1/6 do not sum to exactly one, and "smoothed minus centre" would leak a
// systematic change of sum(phi) into every step. The kernels march along z with the same x-y tiles as
// the fused step (32 columns of which 30 are outputs, BY + 2 rows): every thread keeps three planes
// of its own column in registers and applies the z filters there, one shared-memory plane holds the
// z-filtered values, and the outputs apply the x-y filters from it.
struct PhaseParams {
  int nx, ny, nz;
  long long N;
  double D, lambda, beta, kappa;
  double body[3];    // body force per unit volume (part of F^b)
  double accel[3];   // body acceleration a: F^b also holds rho(phi) a
  double rho_l, drho;  // rho(phi) = rho_l + phi drho
  const uint8_t* mask;  // solid sites (phi frozen, u = 0 there) or null
  Scales sc;
  int zchunk;
};

constexpr int kPhaseRows = 8;  // output rows per CTA of the phase-field kernels

template <class T>
struct PhaseTile {
  static constexpr int ROWS = kPhaseRows + 2;
  static constexpr int SITES = ROWS * 32;
  static constexpr T A0 = T(2) / T(3), A1 = T(1) / T(6);
  // A_x A_y f and the two first differences D_x A_y f, D_y A_x f of the staged plane at site p
  __device__ __forceinline__ static T axay(const T* f) {
    const T r0 = A0 * f[0] + A1 * (f[-1] + f[1]);
    const T rm = A0 * f[-32] + A1 * (f[-33] + f[-31]);
    const T rp = A0 * f[32] + A1 * (f[31] + f[33]);
    return A0 * r0 + A1 * (rm + rp);
  }
  __device__ __forceinline__ static T dxay(const T* f) {
    return A1 * (A0 * (f[1] - f[-1]) + A1 * ((f[-31] - f[-33]) + (f[33] - f[31])));
  }
  __device__ __forceinline__ static T dyax(const T* f) {
    return A1 * (A0 * (f[32] - f[-32]) + A1 * ((f[31] - f[-33]) + (f[33] - f[-31])));
  }
  // L_x A_y f + L_y f: the in-plane part of the Laplacian sum, zero on a constant field
  __device__ __forceinline__ static T lap_xy(const T* f) {
    const T am = A0 * f[-1] + A1 * (f[-33] + f[31]);
    const T a0 = A0 * f[0] + A1 * (f[-32] + f[32]);
    const T ap = A0 * f[1] + A1 * (f[-31] + f[33]);
    return A1 * ((am - a0) + (ap - a0)) + A1 * ((f[-32] - f[0]) + (f[32] - f[0]));
  }
};

// this thread's column of a phase-field kernel tile and its output flag
struct PhaseColumn {
  long long col;  // site index within a plane (periodically wrapped)
  bool out;
  int z0, z1;
  __device__ __forceinline__ PhaseColumn(const PhaseParams& p) {
    const int gx = int(blockIdx.x) * 30 - 1 + int(threadIdx.x);
    const int gy = int(blockIdx.y) * kPhaseRows - 1 + int(threadIdx.y);
    const int sx = ((gx % p.nx) + p.nx) % p.nx, sy = ((gy % p.ny) + p.ny) % p.ny;
    col = (long long)sy * p.nx + sx;
    out = threadIdx.y >= 1 && threadIdx.y <= kPhaseRows && threadIdx.x >= 1 && threadIdx.x <= 30 && gx < p.nx &&
          gy < p.ny;
    z0 = int(blockIdx.z) * p.zchunk;
    z1 = min(p.nz, z0 + p.zchunk);
  }
};

// phi_new from phi, u (decoded from the state) and G, all at time n:
//   phi' = phi - 3 sum_i w_i c_i . V(x + c_i) + 6 D sum_i w_i (phi(x + c_i) - phi(x)),
//   V = phi u + lambda G
// With walls, u is taken as 0 at solid sites and phi is not advanced there (it keeps its value),
// so a wall in contact with one bulk phase exchanges no phi.
template <class S, class T>
__global__ void __launch_bounds__(PhaseTile<T>::SITES) k_phase_advance(const S* __restrict__ st,
                                                                       const T* __restrict__ phi,
                                                                       const T* __restrict__ G,
                                                                       T* __restrict__ phi_new, PhaseParams p) {
  using PT = PhaseTile<T>;
  __shared__ T sm[5][PT::SITES];  // phi, L_z phi, A_z V_x, A_z V_y, D_z V_z of the current plane
  const PhaseColumn c(p);
  const int me = threadIdx.y * 32 + threadIdx.x;
  const long long N = p.N, plane = (long long)p.nx * p.ny;
  const T lam = T(p.lambda), dif6 = T(6) * T(p.D);
  // planes z-1, z, z+1 of this column: phi and V
  T f[3], vx[3], vy[3], vz[3];
  // raw values of the plane after those (prefetched)
  T rph, rux, ruy, ruz, rgx, rgy, rgz;
  auto fetch = [&](int zp) {
    const long long s = (long long)wrap(zp, p.nz) * plane + c.col;  // zp in [-1, nz]
    rph = phi[s];
    if constexpr (Codec<S>::scaled) {
      rux = T(Codec<S>::load(st + N + s) * p.sc.dec[1]);
      ruy = T(Codec<S>::load(st + 2 * N + s) * p.sc.dec[1]);
      ruz = T(Codec<S>::load(st + 3 * N + s) * p.sc.dec[1]);
    } else {
      rux = st[N + s];
      ruy = st[2 * N + s];
      ruz = st[3 * N + s];
    }
    rgx = G[s];
    rgy = G[N + s];
    rgz = G[2 * N + s];
    if (p.mask != nullptr && p.mask[s]) rux = ruy = ruz = T(0);
  };
  auto take = [&](int k) {
    f[k] = rph;
    vx[k] = rph * rux + lam * rgx;
    vy[k] = rph * ruy + lam * rgy;
    vz[k] = rph * ruz + lam * rgz;
  };
  fetch(c.z0 - 1);
  take(0);
  fetch(c.z0);
  take(1);
  fetch(c.z0 + 1);
  for (int z = c.z0; z < c.z1; ++z) {
    take(2);
    if (z + 2 <= c.z1) fetch(z + 2);  // in flight during this plane
    sm[0][me] = f[1];
    sm[1][me] = PT::A1 * ((f[0] - f[1]) + (f[2] - f[1]));
    sm[2][me] = PT::A0 * vx[1] + PT::A1 * (vx[0] + vx[2]);
    sm[3][me] = PT::A0 * vy[1] + PT::A1 * (vy[0] + vy[2]);
    sm[4][me] = PT::A1 * (vz[2] - vz[0]);
    __syncthreads();
    if (c.out) {
      const T div = PT::dxay(sm[2] + me) + PT::dyax(sm[3] + me) + PT::axay(sm[4] + me);
      const T lap = PT::lap_xy(sm[0] + me) + PT::axay(sm[1] + me);
      const long long s = (long long)z * plane + c.col;
      phi_new[s] = (p.mask != nullptr && p.mask[s]) ? f[1] : f[1] - T(3) * div + dif6 * lap;
    }
    __syncthreads();
    f[0] = f[1];
    f[1] = f[2];
    vx[0] = vx[1];
    vx[1] = vx[2];
    vy[0] = vy[1];
    vy[1] = vy[2];
    vz[0] = vz[1];
    vz[1] = vz[2];
  }
}

// force F = mu grad phi + F^b and compression flux G from phi (time n+1):
//   grad phi = 3 (D_x A_y A_z, D_y A_x A_z, D_z A_x A_y) phi, lap phi = 6 (A_x A_y A_z phi - phi),
//   mu = 4 beta phi (phi - 1)(phi - 1/2) - kappa lap phi,  F^b = body + rho(phi) a.
// With a density contrast grad phi is also written (gphi, else null): the fused step forms the
// pressure and viscous-gradient forces from it and the raw moments of the new state.
template <class T>
__global__ void __launch_bounds__(PhaseTile<T>::SITES) k_phase_forces(const T* __restrict__ phi,
                                                                      T* __restrict__ F, T* __restrict__ G,
                                                                      T* __restrict__ gphi, PhaseParams p) {
  using PT = PhaseTile<T>;
  __shared__ T sm[4][PT::SITES];  // A_z phi, D_z phi, phi, L_z phi of the current plane
  const PhaseColumn c(p);
  const int me = threadIdx.y * 32 + threadIdx.x;
  const long long N = p.N, plane = (long long)p.nx * p.ny;
  const T beta4 = T(4) * T(p.beta), kappa = T(p.kappa);
  const T b0 = T(p.body[0]), b1 = T(p.body[1]), b2 = T(p.body[2]);
  const T a0 = T(p.accel[0]), a1 = T(p.accel[1]), a2 = T(p.accel[2]);
  const T rl = T(p.rho_l), dr = T(p.drho);
  auto fetch = [&](int zp) { return phi[(long long)wrap(zp, p.nz) * plane + c.col]; };  // zp in [-1, nz]
  T f0 = fetch(c.z0 - 1), f1 = fetch(c.z0), f2, nxt = fetch(c.z0 + 1);
  for (int z = c.z0; z < c.z1; ++z) {
    f2 = nxt;
    if (z + 2 <= c.z1) nxt = fetch(z + 2);
    sm[0][me] = PT::A0 * f1 + PT::A1 * (f0 + f2);
    sm[1][me] = PT::A1 * (f2 - f0);
    sm[2][me] = f1;
    sm[3][me] = PT::A1 * ((f0 - f1) + (f2 - f1));
    __syncthreads();
    if (c.out) {
      const T gx = T(3) * PT::dxay(sm[0] + me), gy = T(3) * PT::dyax(sm[0] + me), gz = T(3) * PT::axay(sm[1] + me);
      const T lap = T(6) * (PT::lap_xy(sm[2] + me) + PT::axay(sm[3] + me));
      const T mu = beta4 * f1 * (f1 - T(1)) * (f1 - T(0.5)) - kappa * lap;
      const long long s = (long long)z * plane + c.col;
      const T rho = rl + f1 * dr;
      F[s] = mu * gx + (b0 + rho * a0);
      F[N + s] = mu * gy + (b1 + rho * a1);
      F[2 * N + s] = mu * gz + (b2 + rho * a2);
      if (gphi != nullptr) {
        gphi[s] = gx;
        gphi[N + s] = gy;
        gphi[2 * N + s] = gz;
      }
      // phi (1 - phi) / max(|grad phi|, 1e-12)
      const T g2 = gx * gx + gy * gy + gz * gz;
      const T cc = f1 * (T(1) - f1) * rsqrt(g2 > T(1e-24) ? g2 : T(1e-24));
      G[s] = cc * gx;
      G[N + s] = cc * gy;
      G[2 * N + s] = cc * gz;
    }
    __syncthreads();
    f0 = f1;
    f1 = f2;
  }
}

// Force of the initial state with a density contrast: F += F^p + F^nu from the stored p* and
// N = A - u u (internal layout, FP32/FP64 storage), with grad rho = (rho_h - rho_l) grad phi:
//   F^p = -p* cs2 grad rho,  F^nu = -(nu omega / cs2) N . grad rho,  nu = nu(phi), omega = 1/(nu/cs2 + 1/2)
template <class S, class T>
__global__ void k_contrast_init(const S* __restrict__ st, const T* __restrict__ phi, const T* __restrict__ gphi,
                                T* __restrict__ F, long long N, double drho, double nu_l, double dnu) {
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < N; s += (long long)gridDim.x * blockDim.x) {
    const T g0 = T(drho) * gphi[s], g1 = T(drho) * gphi[N + s], g2 = T(drho) * gphi[2 * N + s];
    const T p3 = T(st[s]) * (T(1) / T(3));
    const T nxx = T(st[4 * N + s]), nyy = T(st[5 * N + s]), nzz = T(st[6 * N + s]);
    const T nxy = T(st[7 * N + s]), nxz = T(st[8 * N + s]), nyz = T(st[9 * N + s]);
    const T nu = T(nu_l) + phi[s] * T(dnu);
    const T cnu = T(-3) * nu / (T(3) * nu + T(0.5));
    F[s] += -p3 * g0 + cnu * (nxx * g0 + nxy * g1 + nxz * g2);
    F[N + s] += -p3 * g1 + cnu * (nxy * g0 + nyy * g1 + nyz * g2);
    F[2 * N + s] += -p3 * g2 + cnu * (nxz * g0 + nyz * g1 + nzz * g2);
  }
}

}  // namespace lbf
