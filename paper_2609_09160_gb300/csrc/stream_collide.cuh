// Fused pull-stream-and-collide step of the moment-represented lattice Boltzmann method.
//
// One launch advances the 10-field moment state by one time step (Sec. 2, Eq. (pullLLB) followed
// by Eq. (corr)). Populations are never written to global memory: every site's post-collision
// populations are rebuilt from its stored moments into a shared-memory ring, pulled by the
// neighbours, and folded straight into the new moments.
//
// Work decomposition (GB300: 152 SMs, 228 KB shared memory per SM):
//   * a CTA owns an x-y tile of 30 x BY output columns and marches along z through a chunk of planes;
//   * it has BY+2 warps; warp r holds one row of 32 consecutive sites: the 30 outputs of that row
//     plus the x halo on either side (lanes 0 and 31), and warps 0 and BY+1 are the y halo rows;
//   * per plane every thread loads its site's 10 stored values (coalesced SoA loads), forms the
//     post-collision Hermite coefficients P and the Q populations f_q = w_q [P0 + 3 c.P1 +
//     (9/2) (c c - delta/3) : P2] and writes them to slot (z+1) of a 3-plane ring;
//   * after a barrier the output threads pull f_q(x - c_q) from the ring (planes z-1, z, z+1),
//     sum them pairwise into the new moments, apply the half-force correction and store.
// Halfway bounce-back: where x - c_q is solid the pulled value is the opposite population of x
// itself. A block-wide OR of the solid flags of the three ring planes skips that logic for tiles
// with no wall nearby.
// The conservation sums (sum p*, sum u, sum phi, sum u.u) are accumulated per thread and reduced
// in FP64 across the CTA into one partial per block (deterministic second stage elsewhere).
#pragma once

#include "lattice.cuh"

namespace lbf {

template <class S>
struct ComputeOf {
  using type = float;
};
template <>
struct ComputeOf<double> {
  using type = double;
};

struct FwdParams {
  const void* src;          // state at t (storage type), [10][nz][ny][nx]
  void* dst;                // state at t+1
  const uint8_t* mask;      // [nz][ny][nx], 1 = solid, or null
  const void* force_field;  // compute type [3][nz][ny][nx] or null (added to the uniform force)
  double force[3];          // uniform body force
  double omega;             // single-component relaxation rate 1/tau
  // two-component coupling: phi and the total force at t (sources) and at t+1 (correction)
  const void* phi_old;
  const void* phi_new;
  const void* F_old;
  const void* F_new;
  double rho_l, rho_h, nu_l, nu_h;
  int nx, ny, nz;
  long long N;              // nx*ny*nz
  Scales sc;
  double* partials;         // 8 doubles per block, or null (no reduction this step)
  double* sums;             // 6 final sums, written by the last block to finish
  unsigned* counter;        // blocks done; reset to 0 by the last block
  unsigned* flags;          // bit 0: non-finite or |u|^2 > umax2 seen
  int zchunk;
  float umax2;
};

template <class S, class T>
__device__ __forceinline__ T ld_field(const S* base, long long idx, float dec) {
  if constexpr (Codec<S>::scaled)
    return static_cast<T>(Codec<S>::load(base + idx) * dec);
  else
    return static_cast<T>(Codec<S>::load(base + idx));
}

template <class S, class T>
__device__ __forceinline__ void st_field(S* base, long long idx, T v, float enc) {
  if constexpr (Codec<S>::scaled)
    Codec<S>::store(base + idx, static_cast<float>(v) * enc);
  else
    Codec<S>::store(base + idx, v);
}

// Post-collision Hermite coefficients of one site (the bracket of Eq. (pullLLB) in Hermite form):
//   P0 = p*,  P1 = u + F/(2 rho),  P2 = u u + (1 - omega) N + (u F + F u)/(2 rho)
// where N = a2 - u u is the stored non-equilibrium part and F the force at the site (Eq. guoforce
// projects onto F/rho and (uF + Fu)/rho; half of it enters here).
// Returned pre-scaled for the population formula: q0 = P0 - (3/2) tr P2, b = 3 P1,
// e_aa = (9/2) P2_aa, e_ab = 9 P2_ab (a < b).
template <class T>
struct PostColl {
  T q0, bx, by, bz, exx, eyy, ezz, exy, exz, eyz;
};

template <class T>
__device__ __forceinline__ PostColl<T> post_collision(T p, T ux, T uy, T uz, T nxx, T nyy, T nzz, T nxy,
                                                       T nxz, T nyz, T Fx, T Fy, T Fz, T inv2rho,
                                                       T one_m_omega) {
  const T hx = Fx * inv2rho, hy = Fy * inv2rho, hz = Fz * inv2rho;
  const T pxx = ux * ux + one_m_omega * nxx + T(2) * ux * hx;
  const T pyy = uy * uy + one_m_omega * nyy + T(2) * uy * hy;
  const T pzz = uz * uz + one_m_omega * nzz + T(2) * uz * hz;
  const T pxy = ux * uy + one_m_omega * nxy + (ux * hy + hx * uy);
  const T pxz = ux * uz + one_m_omega * nxz + (ux * hz + hx * uz);
  const T pyz = uy * uz + one_m_omega * nyz + (uy * hz + hy * uz);
  PostColl<T> r;
  r.q0 = p - T(1.5) * (pxx + pyy + pzz);
  r.bx = T(3) * (ux + hx);
  r.by = T(3) * (uy + hy);
  r.bz = T(3) * (uz + hz);
  r.exx = T(4.5) * pxx;
  r.eyy = T(4.5) * pyy;
  r.ezz = T(4.5) * pzz;
  r.exy = T(9) * pxy;
  r.exz = T(9) * pxz;
  r.eyz = T(9) * pyz;
  return r;
}

// f_q and f_opp(q) of one site: w_q (s +/- d) with s = q0 + c.e.c and d = c.b
template <class L, int q, class T>
__device__ __forceinline__ void pop_pair(const PostColl<T>& P, T& fq, T& fo) {
  constexpr int cx = L::cx(q), cy = L::cy(q), cz = L::cz(q);
  T s = P.q0;
  s = sadd<cx * cx>(s, P.exx);
  s = sadd<cy * cy>(s, P.eyy);
  s = sadd<cz * cz>(s, P.ezz);
  s = sadd<cx * cy>(s, P.exy);
  s = sadd<cx * cz>(s, P.exz);
  s = sadd<cy * cz>(s, P.eyz);
  T d;
  if constexpr (cx != 0) {
    d = (cx > 0) ? P.bx : -P.bx;
    d = sadd<cy>(d, P.by);
    d = sadd<cz>(d, P.bz);
  } else if constexpr (cy != 0) {
    d = (cy > 0) ? P.by : -P.by;
    d = sadd<cz>(d, P.bz);
  } else {
    d = (cz > 0) ? P.bz : -P.bz;
  }
  constexpr T w = T(L::w(q));
  fq = w * (s + d);
  fo = w * (s - d);
}

// new raw moments accumulated from pulled populations, pairwise
template <class T>
struct Accum {
  T a0, jx, jy, jz, rxx, ryy, rzz, rxy, rxz, ryz;
};

template <int cx, int cy, int cz, class T>
__device__ __forceinline__ void accumulate_pair(Accum<T>& A, T fq, T fo) {
  const T s = fq + fo, d = fq - fo;
  A.a0 += s;
  A.jx = sadd<cx>(A.jx, d);
  A.jy = sadd<cy>(A.jy, d);
  A.jz = sadd<cz>(A.jz, d);
  A.rxx = sadd<cx * cx>(A.rxx, s);
  A.ryy = sadd<cy * cy>(A.ryy, s);
  A.rzz = sadd<cz * cz>(A.rzz, s);
  A.rxy = sadd<cx * cy>(A.rxy, s);
  A.rxz = sadd<cx * cz>(A.rxz, s);
  A.ryz = sadd<cy * cz>(A.ryz, s);
}

template <int BY>
struct FwdTile {
  static constexpr int ROWS = BY + 2;
  static constexpr int THREADS = 32 * ROWS;
  static constexpr int XOUT = 30;
};

template <class L, class T, int BY, bool MASK>
constexpr size_t fwd_smem_bytes() {
  return size_t(3) * L::Q * FwdTile<BY>::ROWS * 32 * sizeof(T) + (MASK ? size_t(3) * FwdTile<BY>::ROWS * 32 : 0);
}

template <class L, class S, int BY, bool MASK, bool TWO>
__global__ void __launch_bounds__(FwdTile<BY>::THREADS)
    k_stream_collide(const FwdParams a) {
  using T = typename ComputeOf<S>::type;
  constexpr int Q = L::Q;
  constexpr int ROWS = FwdTile<BY>::ROWS;
  constexpr int REST = rest_index<L>();
  constexpr int PLANE = Q * ROWS * 32;  // populations of one ring slot
  static_assert(fwd_smem_bytes<L, T, BY, MASK>() >= 6 * 512 * sizeof(double), "ring too small for the final tree");
  static_assert(FwdTile<BY>::THREADS <= 512, "final tree assumes <= 512 threads");

  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* pop = reinterpret_cast<T*>(smem_raw);
  uint8_t* msk = reinterpret_cast<uint8_t*>(smem_raw + size_t(3) * PLANE * sizeof(T));
  __shared__ double red_s[ROWS][6];

  const S* __restrict__ src = static_cast<const S*>(a.src);
  S* __restrict__ dst = static_cast<S*>(a.dst);
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

  const T one_m_omega = T(1) - T(a.omega);
  const T Fu[3] = {T(a.force[0]), T(a.force[1]), T(a.force[2])};

  // own-site values needed by the output of the plane staged one iteration earlier
  T Fown[3] = {Fu[0], Fu[1], Fu[2]};
  T Fnext[3] = {Fu[0], Fu[1], Fu[2]};
  T inv2rho_own = T(0.5), inv2rho_next = T(0.5);
  T phi_own = T(0), phi_next = T(0);
  bool solid_own = false, solid_next = false;

  auto stage = [&](int zp, int slot) -> bool {
    const int z = wrap(zp, a.nz);
    const long long site = (long long)z * plane + col;
    const T p = ld_field<S, T>(src, site, a.sc.dec[0]);
    const T ux = ld_field<S, T>(src, N + site, a.sc.dec[1]);
    const T uy = ld_field<S, T>(src, 2 * N + site, a.sc.dec[1]);
    const T uz = ld_field<S, T>(src, 3 * N + site, a.sc.dec[1]);
    const T nxx = ld_field<S, T>(src, 4 * N + site, a.sc.dec[2]);
    const T nyy = ld_field<S, T>(src, 5 * N + site, a.sc.dec[2]);
    const T nzz = ld_field<S, T>(src, 6 * N + site, a.sc.dec[2]);
    const T nxy = ld_field<S, T>(src, 7 * N + site, a.sc.dec[2]);
    const T nxz = ld_field<S, T>(src, 8 * N + site, a.sc.dec[2]);
    const T nyz = ld_field<S, T>(src, 9 * N + site, a.sc.dec[2]);
    T F[3] = {Fu[0], Fu[1], Fu[2]};
    T inv2rho = T(0.5);
    T omm = one_m_omega;
    if constexpr (TWO) {
      const T* phi_o = static_cast<const T*>(a.phi_old);
      const T* F_o = static_cast<const T*>(a.F_old);
      const T ph = __ldg(phi_o + site);
      const T rho = T(a.rho_l) + ph * T(a.rho_h - a.rho_l);
      const T nu = T(a.nu_l) + ph * T(a.nu_h - a.nu_l);
      inv2rho = T(0.5) / rho;
      omm = T(1) - T(1) / (T(3) * nu + T(0.5));
      F[0] = __ldg(F_o + site);
      F[1] = __ldg(F_o + N + site);
      F[2] = __ldg(F_o + 2 * N + site);
      if (outcol) {
        const T* phi_n = static_cast<const T*>(a.phi_new);
        const T* F_n = static_cast<const T*>(a.F_new);
        phi_next = __ldg(phi_n + site);
        inv2rho_next = T(0.5) / (T(a.rho_l) + phi_next * T(a.rho_h - a.rho_l));
        Fnext[0] = __ldg(F_n + site);
        Fnext[1] = __ldg(F_n + N + site);
        Fnext[2] = __ldg(F_n + 2 * N + site);
      }
    } else {
      if (ffield != nullptr) {
        F[0] += __ldg(ffield + site);
        F[1] += __ldg(ffield + N + site);
        F[2] += __ldg(ffield + 2 * N + site);
      }
      Fnext[0] = F[0];
      Fnext[1] = F[1];
      Fnext[2] = F[2];
    }
    const PostColl<T> P = post_collision<T>(p, ux, uy, uz, nxx, nyy, nzz, nxy, nxz, nyz, F[0], F[1], F[2],
                                            inv2rho, omm);
    T* ps = pop + slot * PLANE + me;
    static_for<Q>([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      if constexpr (q == REST) {
        ps[q * ROWS * 32] = T(L::w(q)) * P.q0;
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
    solid_next = solid;
    return solid;
  };

  auto shift_own = [&]() {
    Fown[0] = Fnext[0];
    Fown[1] = Fnext[1];
    Fown[2] = Fnext[2];
    inv2rho_own = inv2rho_next;
    phi_own = phi_next;
    solid_own = solid_next;
  };

  T red[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};

  // ring: slot of plane z-1, z, z+1 (rotating)
  int s_m = 0, s_0 = 1, s_p = 2;
  bool any_m = stage(z0 - 1, s_m);
  bool any_0 = stage(z0, s_0);
  shift_own();
  if constexpr (MASK) {
    any_m = __syncthreads_or(any_m);
    any_0 = __syncthreads_or(any_0);
  }
  for (int z = z0; z < z1; ++z) {
    // own values of plane z were shifted in at the end of the previous iteration (or prologue)
    const T Fo0 = Fown[0], Fo1 = Fown[1], Fo2 = Fown[2];
    const T i2r = inv2rho_own;
    const T phio = phi_own;
    const bool solido = solid_own;
    bool any_p = stage(z + 1, s_p);
    if constexpr (MASK)
      any_p = __syncthreads_or(any_p);
    else
      __syncthreads();
    if (outcol && !solido) {
      const bool walls = MASK && (any_m || any_0 || any_p);
      Accum<T> A = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
      const T* base0 = pop + s_0 * PLANE + me;
      A.a0 = base0[REST * ROWS * 32];
      static_for<Q>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        if constexpr (q != REST && q < L::opp(q)) {
          constexpr int o = L::opp(q);
          constexpr int cx = L::cx(q), cy = L::cy(q), cz = L::cz(q);
          // f_q pulled from x - c_q (plane z - cz), f_o from x + c_q (plane z + cz)
          const int slot_q = cz > 0 ? s_m : (cz < 0 ? s_p : s_0);
          const int slot_o = cz > 0 ? s_p : (cz < 0 ? s_m : s_0);
          const int off_q = -cy * 32 - cx;
          const int off_o = cy * 32 + cx;
          T fq = pop[slot_q * PLANE + q * ROWS * 32 + me + off_q];
          T fo = pop[slot_o * PLANE + o * ROWS * 32 + me + off_o];
          if constexpr (MASK) {
            if (walls) {
              if (msk[slot_q * ROWS * 32 + me + off_q]) fq = base0[o * ROWS * 32];
              if (msk[slot_o * ROWS * 32 + me + off_o]) fo = base0[q * ROWS * 32];
            }
          }
          accumulate_pair<cx, cy, cz, T>(A, fq, fo);
        }
      });
      // Eq. (corr): u = a1 + F/(2 rho), a2 = (sum c c f - cs2 a0 delta) + (u F + F u)/(2 rho)
      const T ux = A.jx + Fo0 * i2r, uy = A.jy + Fo1 * i2r, uz = A.jz + Fo2 * i2r;
      const T hx = Fo0 * i2r, hy = Fo1 * i2r, hz = Fo2 * i2r;
      const T third = T(1) / T(3);
      const T a0c = A.a0 * third;
      const T nxx = (A.rxx - a0c) + T(2) * ux * hx - ux * ux;
      const T nyy = (A.ryy - a0c) + T(2) * uy * hy - uy * uy;
      const T nzz = (A.rzz - a0c) + T(2) * uz * hz - uz * uz;
      const T nxy = A.rxy + (ux * hy + hx * uy) - ux * uy;
      const T nxz = A.rxz + (ux * hz + hx * uz) - ux * uz;
      const T nyz = A.ryz + (uy * hz + hy * uz) - uy * uz;
      const long long site = (long long)z * plane + col;
      st_field<S, T>(dst, site, A.a0, a.sc.enc[0]);
      st_field<S, T>(dst, N + site, ux, a.sc.enc[1]);
      st_field<S, T>(dst, 2 * N + site, uy, a.sc.enc[1]);
      st_field<S, T>(dst, 3 * N + site, uz, a.sc.enc[1]);
      st_field<S, T>(dst, 4 * N + site, nxx, a.sc.enc[2]);
      st_field<S, T>(dst, 5 * N + site, nyy, a.sc.enc[2]);
      st_field<S, T>(dst, 6 * N + site, nzz, a.sc.enc[2]);
      st_field<S, T>(dst, 7 * N + site, nxy, a.sc.enc[2]);
      st_field<S, T>(dst, 8 * N + site, nxz, a.sc.enc[2]);
      st_field<S, T>(dst, 9 * N + site, nyz, a.sc.enc[2]);
      const T uu = ux * ux + uy * uy + uz * uz;
      if (!(uu <= T(a.umax2))) atomicOr(a.flags, 1u);
      red[0] += A.a0;
      red[1] += ux;
      red[2] += uy;
      red[3] += uz;
      red[4] += phio;
      red[5] += uu;
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

  if (a.partials != nullptr) {
    double v[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      v[k] = static_cast<double>(red[k]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    }
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < 6; ++k) red_s[row][k] = v[k];
    }
    __syncthreads();
    const long long nb = (long long)gridDim.x * gridDim.y * gridDim.z;
    if (me < 6) {
      double s = 0.0;
      for (int r = 0; r < ROWS; ++r) s += red_s[r][me];
      const long long b = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
      a.partials[b * 8 + me] = s;
    }
    // second stage in the same launch: the last block to finish sums the partials in a fixed
    // order (thread t takes blocks t, t + T, ...; then a fixed tree), so the result is
    // deterministic and a step is a single kernel
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (me == 0) last = atomicAdd(a.counter, 1u) == (unsigned)(nb - 1);
    __syncthreads();
    if (last) {
      __threadfence();
      // fixed-shape tree over 512 slots per quantity, in the (now idle) ring buffer
      constexpr int NT = FwdTile<BY>::THREADS;
      double* tree = reinterpret_cast<double*>(smem_raw);
      for (int i = me; i < 6 * 512; i += NT) tree[i] = 0.0;
      __syncthreads();
      for (int k = 0; k < 6; ++k) {
        double acc = 0.0;
        for (long long b = me; b < nb; b += NT) acc += __ldcg(a.partials + b * 8 + k);
        tree[k * 512 + me] = acc;
      }
      __syncthreads();
      for (int h = 256; h > 0; h >>= 1) {
        for (int i = me; i < 6 * h; i += NT) {
          const int k = i / h, j = i % h;
          tree[k * 512 + j] += tree[k * 512 + j + h];
        }
        __syncthreads();
      }
      if (me < 6) a.sums[me] = tree[me * 512];
      if (me == 0) *a.counter = 0u;
    }
  }
}

}  // namespace lbf
