// Population-form reference step: the same regularized scheme with the Q populations stored in
// HBM instead of the 10 moments (the representation the paper compares against, Sec. 3: 19 or 27
// fields per buffer instead of 10).
//
// The buffers hold the populations f(x, t) after streaming (the state of the population form of
// Eq. (pullLB)), [Q][nz][ny][nx]. One launch per step, one thread per site (x-rows of 256 sites
// per block, one block row per (y, z)):
//   * read the site's own Q populations and take their Hermite moments with the half-force shift
//     of Eq. (corr) -> (p*, u, A) at t;
//   * collide from those moments (the regularized collision depends only on them, Eqs. reqtfeq
//     and guoforce) and push f*_i to x + c_i, or back to the site itself as f_opp(i) where x + c_i
//     is solid (halfway bounce-back).
// It moves 2 Q sizeof(T) bytes per site (152 B for D3Q19 FP32) against 80 B for the moment
// representation, and needs no shared memory or halo recomputation. Moments are read back from
// the stored populations directly.
#pragma once

#include "stream_collide.cuh"

namespace lbf {

struct PopParams {
  const void* src;          // post-collision populations at t, [Q][nz][ny][nx]
  void* dst;                // at t+1
  void* mom;                // moments kernel: internal moment state [10][nz][ny][nx] (solid sites kept)
  const uint8_t* mask;      // [nz][ny][nx], 1 = solid, or null
  const void* force_field;  // compute type [3][nz][ny][nx] or null (added to the uniform force)
  double force[3];
  float force_f[3];
  double omega;
  float omega_f;
  int nx, ny, nz;
  long long N;
  unsigned* flags;   // bit 0: non-finite value or |u|^2 > umax2
  float umax2;
};

constexpr int kPopThreads = 256;

// this thread's site of a population kernel launched on pop_grid(): false outside the lattice
__device__ __forceinline__ bool pop_site(const PopParams& p, int& x, int& y, int& z, long long& s) {
  x = blockIdx.x * kPopThreads + threadIdx.x;
  y = blockIdx.y;
  z = blockIdx.z;
  s = ((long long)z * p.ny + y) * p.nx + x;
  return x < p.nx;
}

// raw moments (a0, a1, sum (c c) f) of a site's own populations
template <class L, class T>
__device__ __forceinline__ Accum<T> pop_own_moments(const T* __restrict__ f, long long s, long long N) {
  constexpr int REST = rest_index<L>();
  Accum<T> A = {__ldg(f + REST * N + s), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
  static_for<L::Q>([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    if constexpr (q != REST && q < L::opp(q)) {
      const T fq = __ldg(f + q * N + s);
      const T fo = __ldg(f + L::opp(q) * N + s);
      accumulate_pair<L::cx(q), L::cy(q), L::cz(q), T>(A, fq, fo, T(1));
    }
  });
  return A;
}

template <class T, bool FF>
__device__ __forceinline__ void pop_force(const PopParams& p, long long s, T& Fx, T& Fy, T& Fz) {
  Fx = pick<T>(p.force[0], p.force_f[0]);
  Fy = pick<T>(p.force[1], p.force_f[1]);
  Fz = pick<T>(p.force[2], p.force_f[2]);
  if constexpr (FF) {
    const T* ff = static_cast<const T*>(p.force_field);
    Fx += __ldg(ff + s);
    Fy += __ldg(ff + p.N + s);
    Fz += __ldg(ff + 2 * p.N + s);
  }
}

// Eq. (corr) at one site: raw moments -> stored (p*, u, N = A - u u)
template <class T>
struct PopMoments {
  T p, ux, uy, uz, nxx, nyy, nzz, nxy, nxz, nyz;
};

template <class T>
__device__ __forceinline__ PopMoments<T> pop_correct(const Accum<T>& A, T Fx, T Fy, T Fz) {
  const T hx = Fx * T(0.5), hy = Fy * T(0.5), hz = Fz * T(0.5);
  PopMoments<T> m;
  m.p = A.a0;
  m.ux = A.jx + hx;
  m.uy = A.jy + hy;
  m.uz = A.jz + hz;
  const T a0c = A.a0 * (T(1) / T(3));
  m.nxx = (A.rxx - a0c) + T(2) * m.ux * hx - m.ux * m.ux;
  m.nyy = (A.ryy - a0c) + T(2) * m.uy * hy - m.uy * m.uy;
  m.nzz = (A.rzz - a0c) + T(2) * m.uz * hz - m.uz * m.uz;
  m.nxy = A.rxy + (m.ux * hy + hx * m.uy) - m.ux * m.uy;
  m.nxz = A.rxz + (m.ux * hz + hx * m.uz) - m.ux * m.uz;
  m.nyz = A.ryz + (m.uy * hz + hy * m.uz) - m.uy * m.uz;
  return m;
}

// target of population q of site (x, y, z): x + c_q (periodic)
template <int cx, int cy, int cz>
__device__ __forceinline__ long long pop_target(int x, int y, int z, const PopParams& p) {
  const int xt = cx == 0 ? x : wrap(x + cx, p.nx);
  const int yt = cy == 0 ? y : wrap(y + cy, p.ny);
  const int zt = cz == 0 ? z : wrap(z + cz, p.nz);
  return ((long long)zt * p.ny + yt) * p.nx + xt;
}

// one time step: moments of the own populations, collision, push (halfway bounce-back)
template <class L, class T, bool MASK, bool FF>
__global__ void __launch_bounds__(kPopThreads) k_pop_step(const PopParams p) {
  const T* __restrict__ f = static_cast<const T*>(p.src);
  T* __restrict__ out = static_cast<T*>(p.dst);
  const T omm = T(1) - pick<T>(p.omega, p.omega_f);
  const long long N = p.N;
  int x, y, z;
  long long s;
  if (pop_site(p, x, y, z, s)) {
    if (MASK && __ldg(p.mask + s) != 0) return;  // solid sites hold no populations
    T Fx, Fy, Fz;
    pop_force<T, FF>(p, s, Fx, Fy, Fz);
    const PopMoments<T> m = pop_correct(pop_own_moments<L, T>(f, s, N), Fx, Fy, Fz);
    const T uu = m.ux * m.ux + m.uy * m.uy + m.uz * m.uz;
    if (!(uu <= T(p.umax2))) atomicOr(p.flags, 1u);
    const PostColl<T> P =
        post_collision<T>(m.p, m.ux, m.uy, m.uz, m.nxx, m.nyy, m.nzz, m.nxy, m.nxz, m.nyz, Fx, Fy, Fz, T(0.5), omm);
    auto push = [&](auto qc, T v) {
      constexpr int q = decltype(qc)::value;
      constexpr int cx = L::cx(q), cy = L::cy(q), cz = L::cz(q);
      if constexpr (cx == 0 && cy == 0 && cz == 0) {
        out[q * N + s] = v;
      } else {
        const long long t = pop_target<cx, cy, cz>(x, y, z, p);
        if (MASK && __ldg(p.mask + t) != 0)
          out[L::opp(q) * N + s] = v;  // halfway bounce-back: returns to the site reversed
        else
          out[q * N + t] = v;
      }
    };
    static_for<L::Q>([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      constexpr int REST = rest_index<L>();
      if constexpr (q == REST) {
        push(qc, T(L::w(q)) * P.q0);
      } else if constexpr (q < L::opp(q)) {
        T gq, go;
        pop_pair<L, q, T>(P, gq, go);
        push(qc, T(L::w(q)) * gq);
        push(std::integral_constant<int, L::opp(q)>{}, T(L::w(q)) * go);
      }
    });
  }
}

// populations f(x, t) of every fluid site from the internal moment state p.mom: the truncated
// Hermite expansion with the Eq. (corr) shift undone (a1 = u - F/2, a2 = A - (uF + Fu)/2, rho = 1)
template <class L, class T, bool FF>
__global__ void __launch_bounds__(kPopThreads) k_pop_from_moments(const PopParams p) {
  const T* __restrict__ m = static_cast<const T*>(p.mom);
  T* __restrict__ out = static_cast<T*>(p.dst);
  const long long N = p.N;
  int x, y, z;
  long long s;
  if (pop_site(p, x, y, z, s)) {
    T Fx, Fy, Fz;
    pop_force<T, FF>(p, s, Fx, Fy, Fz);
    // post_collision with -F and omega = 1 gives P1 = u - F/2 and P2 = u u + N - (uF + Fu)/2
    const PostColl<T> P = post_collision<T>(m[s], m[N + s], m[2 * N + s], m[3 * N + s], m[4 * N + s], m[5 * N + s],
                                            m[6 * N + s], m[7 * N + s], m[8 * N + s], m[9 * N + s], -Fx, -Fy, -Fz,
                                            T(0.5), T(1));
    static_for<L::Q>([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      constexpr int REST = rest_index<L>();
      if constexpr (q == REST) {
        out[q * N + s] = T(L::w(q)) * P.q0;
      } else if constexpr (q < L::opp(q)) {
        T gq, go;
        pop_pair<L, q, T>(P, gq, go);
        out[q * N + s] = T(L::w(q)) * gq;
        out[L::opp(q) * N + s] = T(L::w(q)) * go;
      }
    });
  }
}

// internal moment state (p*, u, N = A - u u) of every fluid site from its populations; solid sites
// of p.mom keep their values
template <class L, class T, bool MASK, bool FF>
__global__ void __launch_bounds__(kPopThreads) k_pop_moments(const PopParams p) {
  const T* __restrict__ f = static_cast<const T*>(p.src);
  T* __restrict__ m = static_cast<T*>(p.mom);
  const long long N = p.N;
  int x, y, z;
  long long s;
  if (pop_site(p, x, y, z, s)) {
    if (MASK && __ldg(p.mask + s) != 0) return;
    T Fx, Fy, Fz;
    pop_force<T, FF>(p, s, Fx, Fy, Fz);
    const PopMoments<T> v = pop_correct(pop_own_moments<L, T>(f, s, N), Fx, Fy, Fz);
    m[s] = v.p;
    m[N + s] = v.ux;
    m[2 * N + s] = v.uy;
    m[3 * N + s] = v.uz;
    m[4 * N + s] = v.nxx;
    m[5 * N + s] = v.nyy;
    m[6 * N + s] = v.nzz;
    m[7 * N + s] = v.nxy;
    m[8 * N + s] = v.nxz;
    m[9 * N + s] = v.nyz;
  }
}

}  // namespace lbf
