// Discrete adjoint of one fused step (the paper has no adjoint; this is the exact transpose of
// the linearised single-component step of stream_collide.cuh, in the public parametrisation
// M = (p*, u, A), A = a2 the total second Hermite coefficient).
//
// Forward map, per output site x:  P(y) = collide(M_t(y), F(y)) at every source y = x - c_q,
// f_q(x) = w_q H_q . P(x - c_q) (or the bounce-back of x itself), a(x) = sum_q H_q f_q(x),
// M_{t+1}(x) = correct(a(x), F(x)) with Eq. (corr).
// Adjoint, per site, with lambda' = dL/dM_{t+1} and Lam the full symmetric form of lambda'_A
// (off-diagonal stored values halved):
//   x side:  mu0 = lambda'_p,  mu2 = Lam,  mu1 = g = lambda'_u + Lam F / rho,
//            dL/dF(x) += g / (2 rho) + Lam u' / rho,
//            nu_q(x) = mu0 + c_q . mu1 + (c_q c_q - delta/3) : mu2   (= dL/df_q(x));
//   y side:  nu~_q(y) = nu_q(y + c_q), or nu_opp(q)(y) when y + c_q is solid (bounce-back),
//            pi0 = sum w nu~, pi1 = 3 sum w c nu~, pi2 = (9/2) sum w (c c - delta/3) nu~,
//            lambda_p = pi0,  lambda_u = pi1 + 2 omega pi2 u + pi2 F / rho,
//            lambda_A = (1 - omega) pi2 (stored off-diagonals doubled),
//            dL/dF(y) += pi1 / (2 rho) + pi2 u / rho.
// The kernel has the same z-marching shape as the forward one with the pull direction
// reversed: staged values are nu_q(x) (the weight w_q is applied in the gather sums) and the
// gather reads y + c_q.
#pragma once

#include "stream_collide.cuh"

namespace lbf {

struct AdjParams {
  const void* state_t;    // storage type, internal layout
  const void* state_t1;
  const void* lam_in;     // compute type, public layout [10][N]
  void* lam_out;
  double* grad_force;     // [3][N] FP64, accumulated
  const uint8_t* mask;
  const void* force_field;
  double force[3];
  double omega;
  int nx, ny, nz;
  long long N;
  Scales sc;
  int zchunk;
};

// adds the pair (g_q, g_opp(q)) of direction c with weight w like accumulate_pair, but the diagonal
// second moments directly in traceless form, sum w (c_a c_a - 1/3) s: an adjoint field with a large
// isotropic part would otherwise lose its traceless part to the cancellation sum w c_a^2 s - a0 / 3
template <int cx, int cy, int cz, class T>
__device__ __forceinline__ void accumulate_pair_traceless(Accum<T>& A, T gq, T go, T w) {
  const T s = gq + go, d = gq - go;
  A.a0 = fma(w, s, A.a0);
  A.jx = sfma<cx>(A.jx, w, d);
  A.jy = sfma<cy>(A.jy, w, d);
  A.jz = sfma<cz>(A.jz, w, d);
  A.rxx = fma(w * T(cx * cx * 3 - 1) * T(1.0 / 3.0), s, A.rxx);
  A.ryy = fma(w * T(cy * cy * 3 - 1) * T(1.0 / 3.0), s, A.ryy);
  A.rzz = fma(w * T(cz * cz * 3 - 1) * T(1.0 / 3.0), s, A.rzz);
  A.rxy = sfma<cx * cy>(A.rxy, w, s);
  A.rxz = sfma<cx * cz>(A.rxz, w, s);
  A.ryz = sfma<cy * cz>(A.ryz, w, s);
}

template <class L, class S, int BY, bool MASK>
__global__ void __launch_bounds__(FwdTile<BY>::THREADS)
    k_adjoint(const AdjParams a) {
  using T = typename ComputeOf<S>::type;
  constexpr int Q = L::Q;
  constexpr int ROWS = FwdTile<BY>::ROWS;
  constexpr int REST = rest_index<L>();
  constexpr int PLANE = Q * ROWS * 32;

  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* nus = reinterpret_cast<T*>(smem_raw);
  uint8_t* msk = reinterpret_cast<uint8_t*>(smem_raw + size_t(3) * PLANE * sizeof(T));

  const S* __restrict__ st0 = static_cast<const S*>(a.state_t);
  const S* __restrict__ st1 = static_cast<const S*>(a.state_t1);
  const T* __restrict__ lin = static_cast<const T*>(a.lam_in);
  T* __restrict__ lout = static_cast<T*>(a.lam_out);
  const T* __restrict__ ffield = static_cast<const T*>(a.force_field);

  const int lane = threadIdx.x, row = threadIdx.y;
  const int gx = blockIdx.x * FwdTile<BY>::XOUT - 1 + lane;
  const int gy = blockIdx.y * BY - 1 + row;
  const int sx = ((gx % a.nx) + a.nx) % a.nx;
  const int sy = ((gy % a.ny) + a.ny) % a.ny;
  const bool outcol = lane >= 1 && lane <= FwdTile<BY>::XOUT && row >= 1 && row <= BY && gx < a.nx && gy < a.ny;
  const long long plane = (long long)a.nx * a.ny;
  const long long col = (long long)sy * a.nx + sx;
  const long long N = a.N;
  const int z0 = blockIdx.z * a.zchunk;
  const int z1 = min(a.nz, z0 + a.zchunk);
  const int me = row * 32 + lane;
  const T omega = T(a.omega);
  const T rho = T(1);
  const T inv_rho = T(1) / rho;

  // own-site carry from the staged plane to its output one iteration later
  T Fn[3] = {T(0), T(0), T(0)}, Fo[3];
  T gfx_n[3] = {T(0), T(0), T(0)}, gfx_o[3];
  bool solid_n = false, solid_o;

  auto stage = [&](int zp, int slot) -> bool {
    const int z = wrap(zp, a.nz);
    const long long site = (long long)z * plane + col;
    T F[3] = {T(a.force[0]), T(a.force[1]), T(a.force[2])};
    if (ffield != nullptr) {
      F[0] += __ldg(ffield + site);
      F[1] += __ldg(ffield + N + site);
      F[2] += __ldg(ffield + 2 * N + site);
    }
    const T ux = ld_field<S, T>(st1, N + site, a.sc.dec[1]);
    const T uy = ld_field<S, T>(st1, 2 * N + site, a.sc.dec[1]);
    const T uz = ld_field<S, T>(st1, 3 * N + site, a.sc.dec[1]);
    const T lp = __ldg(lin + site);
    const T lux = __ldg(lin + N + site), luy = __ldg(lin + 2 * N + site), luz = __ldg(lin + 3 * N + site);
    const T Lxx = __ldg(lin + 4 * N + site), Lyy = __ldg(lin + 5 * N + site), Lzz = __ldg(lin + 6 * N + site);
    const T Sxy = __ldg(lin + 7 * N + site), Sxz = __ldg(lin + 8 * N + site), Syz = __ldg(lin + 9 * N + site);
    const T Lxy = T(0.5) * Sxy, Lxz = T(0.5) * Sxz, Lyz = T(0.5) * Syz;
    // g = lambda_u + Lam F / rho
    const T gx_ = lux + (Lxx * F[0] + Lxy * F[1] + Lxz * F[2]) * inv_rho;
    const T gy_ = luy + (Lxy * F[0] + Lyy * F[1] + Lyz * F[2]) * inv_rho;
    const T gz_ = luz + (Lxz * F[0] + Lyz * F[1] + Lzz * F[2]) * inv_rho;
    gfx_n[0] = T(0.5) * gx_ * inv_rho + (Lxx * ux + Lxy * uy + Lxz * uz) * inv_rho;
    gfx_n[1] = T(0.5) * gy_ * inv_rho + (Lxy * ux + Lyy * uy + Lyz * uz) * inv_rho;
    gfx_n[2] = T(0.5) * gz_ * inv_rho + (Lxz * ux + Lyz * uy + Lzz * uz) * inv_rho;
    Fn[0] = F[0];
    Fn[1] = F[1];
    Fn[2] = F[2];
    // nu_q = (mu0 - tr Lam / 3) + c.g + c.Lam.c
    PostColl<T> P;
    P.q0 = lp - (Lxx + Lyy + Lzz) * (T(1) / T(3));
    P.bx = gx_;
    P.by = gy_;
    P.bz = gz_;
    P.exx = Lxx;
    P.eyy = Lyy;
    P.ezz = Lzz;
    P.exy = Sxy;
    P.exz = Sxz;
    P.eyz = Syz;
    T* ps = nus + slot * PLANE + me;
    static_for<Q>([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      if constexpr (q == REST) {
        ps[q * ROWS * 32] = P.q0;
      } else if constexpr (q < L::opp(q)) {
        T fq, fo;
        pop_pair<L, q, T>(P, fq, fo);
        ps[q * ROWS * 32] = fq;
        ps[L::opp(q) * ROWS * 32] = fo;
      }
    });
    bool solid = false;
    if constexpr (MASK) {
      solid = __ldg(a.mask + site) != 0;
      msk[slot * ROWS * 32 + me] = solid ? 1 : 0;
    }
    solid_n = solid;
    return solid;
  };
  auto shift_own = [&]() {
    for (int k = 0; k < 3; ++k) {
      Fo[k] = Fn[k];
      gfx_o[k] = gfx_n[k];
    }
    solid_o = solid_n;
  };

  int s_m = 0, s_0 = 1, s_p = 2;
  bool any_m = stage(z0 - 1, s_m);
  bool any_0 = stage(z0, s_0);
  shift_own();
  if constexpr (MASK) {
    any_m = __syncthreads_or(any_m);
    any_0 = __syncthreads_or(any_0);
  }
  for (int z = z0; z < z1; ++z) {
    const T F0 = Fo[0], F1 = Fo[1], F2 = Fo[2];
    const T gx0 = gfx_o[0], gx1 = gfx_o[1], gx2 = gfx_o[2];
    const bool solido = solid_o;
    bool any_p = stage(z + 1, s_p);
    if constexpr (MASK)
      any_p = __syncthreads_or(any_p);
    else
      __syncthreads();
    if (outcol) {
      const long long site = (long long)z * plane + col;
      if (solido) {
        for (int k = 0; k < 10; ++k) lout[k * N + site] = lin[k * N + site];
      } else {
        const bool walls = MASK && (any_m || any_0 || any_p);
        Accum<T> A = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
        const T* base0 = nus + s_0 * PLANE + me;
        A.a0 = T(L::w(REST)) * base0[REST * ROWS * 32];
        // the rest population's share of the traceless diagonal: w_0 (0 - 1/3) nu_0
        A.rxx = A.a0 * T(-1.0 / 3.0);
        A.ryy = A.rxx;
        A.rzz = A.rxx;
        static_for<Q>([&](auto qc) {
          constexpr int q = decltype(qc)::value;
          if constexpr (q != REST && q < L::opp(q)) {
            constexpr int o = L::opp(q);
            constexpr int cx = L::cx(q), cy = L::cy(q), cz = L::cz(q);
            // nu_q from y + c_q (plane z + cz), nu_o from y - c_q (plane z - cz)
            const int slot_q = cz > 0 ? s_p : (cz < 0 ? s_m : s_0);
            const int slot_o = cz > 0 ? s_m : (cz < 0 ? s_p : s_0);
            const int off_q = cy * 32 + cx;
            const int off_o = -cy * 32 - cx;
            T gq = nus[slot_q * PLANE + q * ROWS * 32 + me + off_q];
            T go = nus[slot_o * PLANE + o * ROWS * 32 + me + off_o];
            if constexpr (MASK) {
              if (walls) {
                if (msk[slot_q * ROWS * 32 + me + off_q]) gq = base0[o * ROWS * 32];
                if (msk[slot_o * ROWS * 32 + me + off_o]) go = base0[q * ROWS * 32];
              }
            }
            accumulate_pair_traceless<cx, cy, cz, T>(A, gq, go, T(L::w(q)));
          }
        });
        const T pi0 = A.a0;
        const T p1x = T(3) * A.jx, p1y = T(3) * A.jy, p1z = T(3) * A.jz;
        const T qxx = T(4.5) * A.rxx, qyy = T(4.5) * A.ryy, qzz = T(4.5) * A.rzz;
        const T qxy = T(4.5) * A.rxy, qxz = T(4.5) * A.rxz, qyz = T(4.5) * A.ryz;
        const T ux = ld_field<S, T>(st0, N + site, a.sc.dec[1]);
        const T uy = ld_field<S, T>(st0, 2 * N + site, a.sc.dec[1]);
        const T uz = ld_field<S, T>(st0, 3 * N + site, a.sc.dec[1]);
        const T qux = qxx * ux + qxy * uy + qxz * uz;
        const T quy = qxy * ux + qyy * uy + qyz * uz;
        const T quz = qxz * ux + qyz * uy + qzz * uz;
        const T qFx = qxx * F0 + qxy * F1 + qxz * F2;
        const T qFy = qxy * F0 + qyy * F1 + qyz * F2;
        const T qFz = qxz * F0 + qyz * F1 + qzz * F2;
        const T omm = T(1) - omega;
        lout[site] = pi0;
        lout[N + site] = p1x + T(2) * omega * qux + qFx * inv_rho;
        lout[2 * N + site] = p1y + T(2) * omega * quy + qFy * inv_rho;
        lout[3 * N + site] = p1z + T(2) * omega * quz + qFz * inv_rho;
        lout[4 * N + site] = omm * qxx;
        lout[5 * N + site] = omm * qyy;
        lout[6 * N + site] = omm * qzz;
        lout[7 * N + site] = T(2) * omm * qxy;
        lout[8 * N + site] = T(2) * omm * qxz;
        lout[9 * N + site] = T(2) * omm * qyz;
        double* g = a.grad_force;
        g[site] += static_cast<double>(gx0 + T(0.5) * p1x * inv_rho + qux * inv_rho);
        g[N + site] += static_cast<double>(gx1 + T(0.5) * p1y * inv_rho + quy * inv_rho);
        g[2 * N + site] += static_cast<double>(gx2 + T(0.5) * p1z * inv_rho + quz * inv_rho);
      }
    }
    shift_own();
    __syncthreads();
    const int t = s_m;
    s_m = s_0;
    s_0 = s_p;
    s_p = t;
    any_m = any_0;
    any_0 = any_p;
  }
}

}  // namespace lbf
