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
//   * per plane one elected thread loads the 10 stored fields of the whole patch with a TMA box
//     into a two-stage shared-memory buffer (the y-halo warps wait for it, see below); every thread
//     forms the post-collision Hermite coefficients P of its site and the Q populations
//     f_q / w_q = P0 + 3 c.P1 + (9/2) (c c - delta/3) : P2 and writes them to a ring split by c_z
//     (the axial directions stay in registers);
//   * after a barrier the output threads pull f_q(x - c_q) from planes z-1, z, z+1, sum them
//     pairwise with the weights w_q into the new moments, apply the half-force correction and
//     store;
//   * during the outputs the idle y-halo warps wait for the next plane's TMA box, so the next
//     iteration starts without any thread polling the mbarrier.
// Halfway bounce-back: where x - c_q is solid the pulled value is the opposite population of x
// itself. A block-wide OR of the solid flags of the three ring planes skips that logic for tiles
// with no wall nearby.
// The conservation sums (sum p*, sum u, sum phi, sum u.u) are accumulated per thread, reduced in
// FP64 across the CTA into one partial per block, and summed in a fixed order by the last block.
#pragma once

#include "lattice.cuh"
#include "tma.cuh"

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
  void* F_new;              // density contrast: read (F^s + F^b) and rewritten with the total force
  const void* grad_phi;     // density contrast: grad phi^{n+1} [3][nz][ny][nx]
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
  uint32_t salt;            // per-step word mixed into the stochastic rounding of 16-bit storage
  // output rows of this launch: y_begin .. y_begin + y_rows - 1, taken mod ny (y_rows = 0: all ny
  // rows from 0). The blocks' partial sums go to partials[block_base + block]; final_blocks > 0:
  // launches that run concurrently share the block counter, and the last of their final_blocks
  // blocks to finish adds partials 0 .. final_blocks - 1 (0: this launch alone, block_base + blocks)
  int y_begin, y_rows;
  long long block_base;
  long long final_blocks;
  // FP32 copies of the double scalars above (set_fp32_copies), read by the FP32-compute kernels
  float force_f[3], omega_f, rho_l_f, drho_f, nu_l_f, dnu_f;
};

inline void set_fp32_copies(FwdParams& a) {
  for (int k = 0; k < 3; ++k) a.force_f[k] = float(a.force[k]);
  a.omega_f = float(a.omega);
  a.rho_l_f = float(a.rho_l);
  a.drho_f = float(a.rho_h - a.rho_l);
  a.nu_l_f = float(a.nu_l);
  a.dnu_f = float(a.nu_h - a.nu_l);
}

// a kernel scalar in the compute type: the FP64 value for FP64 compute, else its FP32 copy
template <class T>
__device__ __forceinline__ T pick(double d, float f) {
  if constexpr (std::is_same<T, double>::value)
    return d;
  else
    return f;
}

template <class S, class T>
__device__ __forceinline__ T ld_field(const S* base, long long idx, float dec) {
  if constexpr (Codec<S>::scaled)
    return static_cast<T>(Codec<S>::load(base + idx) * dec);
  else
    return static_cast<T>(Codec<S>::load(base + idx));
}

// one field of a time step's output: 16-bit storage is scaled and rounded stochastically with the
// next word of the site's random sequence rs
template <class S, bool NEAREST, class T>
__device__ __forceinline__ void st_field(S* base, long long idx, T v, float enc, uint32_t& rs) {
  if constexpr (Codec<S>::scaled && NEAREST) {
    Codec<S>::store(base + idx, static_cast<float>(v) * enc);
  } else if constexpr (Codec<S>::scaled) {
    rs = lcg_next(rs);
    Codec<S>::store_sr(base + idx, static_cast<float>(v) * enc, rs);
  } else {
    Codec<S>::store(base + idx, v);
  }
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

// f_q / w_q and f_opp(q) / w_q of one site: s +/- d with s = q0 + c.e.c and d = c.b. The weight
// w_q (equal for q and opp(q)) is applied where the pulled populations are summed.
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
  fq = s + d;
  fo = s - d;
}

// ---------------------------------------------------------------------------------------------
// D3Q27h (Sec. 2, complete Hermite basis with the recursive closure). For the multi-index
// m = (mx, my, mz) in {0,1,2}^3 (how often each axis occurs in the tensor index) the
// post-collision coefficient is
//   P_m = u^m + (1 - omega) a_neq(m) + S_m / 2,   P_0 = p*,
// with a_neq(m) = N for |m| = 2 and, for |m| >= 3, the sum over index pairs of N times the u's of
// the other indices (the closure), and S_m / 2 the sum over index positions of h = F / (2 rho)
// times the u's of the other indices (the Guo source to the same order). The basis functions are
// h_mx(c_x) h_my(c_y) h_mz(c_z), h_0 = 1, h_1 = c, h_2 = c^2 - 1/3, normalised by
// prod m_a! cs2^m_a, so f_q / w_q = sum_m H_m(c_q) P_m / norm_m is three one-axis contractions in
// which the normalisation folds into the constants: per axis the value at c = 0 is
// P_0 - 1.5 P_2 and at c = +/-1 it is P_0 + 3 P_2 +/- 3 P_1 (indices: the multiplicity of that
// axis). Truncated at |m| <= 2 this is the second-order post_collision / pop_pair above.
// The kernel evaluates this sum in the factorised form below instead of forming the 27 P_m.
// f_q / w_q of all 27 directions in cube order, q = 9 (c_z + 1) + 3 (c_y + 1) + (c_x + 1).
// Every part of sum_m H_m(c) P_m / norm_m factorises over the axes: with the per-axis series
//   phi_a(c)   = sum_k h_k(c) u_a^k / norm_k = 1 + 3 c u_a + 4.5 (c^2 - 1/3) u_a^2
//   sig_a(c)   = h_a d(phi_a)/du_a,   del_a(c) = d(phi_a)/du_a = 3 c + 9 (c^2 - 1/3) u_a,
//   nu_a(c)    = (1/2) d2(phi_a)/du_a2 = 4.5 (c^2 - 1/3),
// the equilibrium part is p* + phi_x phi_y phi_z - 1, the Guo part replaces one factor phi_a by
// sig_a, and the closure part is sum_a N_aa nu_a (other phi) + sum_(a<b) N_ab del_a del_b phi_c
// (the coefficients P_m above summed over the basis, regrouped by axis).
template <class T>
__device__ __forceinline__ void full_populations(T p, const T (&u)[3], const T (&h)[3], const T (&Nt)[3][3], T omm,
                                                 T (&g)[27]) {
  // ps = phi - 1 (small): the equilibrium part p* + prod(1 + ps) - 1 is accumulated as
  // ps_x + phi_x (ps_y + phi_y ps_z), so no O(1) term is ever cancelled (FP32 keeps the deviations)
  T ph[3][3], ps[3][3], sg[3][3], dl[3][3];  // [axis][c + 1]
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const T u2 = u[a] * u[a];
    ps[a][1] = T(-1.5) * u2;
    const T e = T(3) * u2;
    ps[a][2] = e + T(3) * u[a];
    ps[a][0] = e - T(3) * u[a];
#pragma unroll
    for (int c = 0; c < 3; ++c) ph[a][c] = T(1) + ps[a][c];
    const T hu = T(6) * h[a] * u[a];  // 4.5 * (2/3) * 2 h u, and -1.5 * 2 h u = -hu / 2
    sg[a][1] = T(-0.5) * hu;
    sg[a][2] = hu + T(3) * h[a];
    sg[a][0] = hu - T(3) * h[a];
    dl[a][1] = T(-3) * u[a];
    dl[a][2] = T(3) + T(6) * u[a];
    dl[a][0] = T(-3) + T(6) * u[a];
  }
  const T nu0 = T(-1.5), nu1 = T(3);  // nu_a at c = 0 and c = +/-1
  // per (c_x, c_y) column the 27 values are g = K0 + K1 ps_z + K2 sig_z + K3 nu_z + K4 del_z
  const T nxx0 = Nt[0][0] * nu0, nxx1 = Nt[0][0] * nu1, nyy0 = Nt[1][1] * nu0, nyy1 = Nt[1][1] * nu1;
  const T oz = omm * Nt[2][2];
#pragma unroll
  for (int cy = 0; cy < 3; ++cy)
#pragma unroll
    for (int cx = 0; cx < 3; ++cx) {
      const T A = ph[0][cx] * ph[1][cy];
      const T Exy = p + (ps[0][cx] + ph[0][cx] * ps[1][cy]);  // p* + phi_x phi_y - 1
      const T Bs = sg[0][cx] * ph[1][cy] + ph[0][cx] * sg[1][cy];
      const T Bn = (cx == 1 ? nxx0 : nxx1) * ph[1][cy] + (cy == 1 ? nyy0 : nyy1) * ph[0][cx] +
                   Nt[0][1] * (dl[0][cx] * dl[1][cy]);
      const T t = Bs + omm * Bn;
      const T K0 = Exy + t, K1 = A + t, K3 = oz * A;
      const T K4 = omm * (Nt[0][2] * (dl[0][cx] * ph[1][cy]) + Nt[1][2] * (ph[0][cx] * dl[1][cy]));
#pragma unroll
      for (int cz = 0; cz < 3; ++cz)
        g[9 * cz + 3 * cy + cx] = K0 + K1 * ps[2][cz] + A * sg[2][cz] + K3 * (cz == 1 ? nu0 : nu1) + K4 * dl[2][cz];
    }
}

// new raw moments accumulated from pulled populations, pairwise
template <class T>
struct Accum {
  T a0, jx, jy, jz, rxx, ryy, rzz, rxy, rxz, ryz;
};

// acc + C w v for a compile-time C in {-1, 0, 1}
template <int C, class T>
__device__ __forceinline__ T sfma(T acc, T w, T v) {
  if constexpr (C > 0)
    return fma(w, v, acc);
  else if constexpr (C < 0)
    return fma(-w, v, acc);
  else
    return acc;
}

// adds the pair (f_q, f_opp(q)) = w (gq, go) of direction c = (cx, cy, cz) with weight w
template <int cx, int cy, int cz, class T>
__device__ __forceinline__ void accumulate_pair(Accum<T>& A, T gq, T go, T w) {
  const T s = gq + go, d = gq - go;
  A.a0 = fma(w, s, A.a0);
  A.jx = sfma<cx>(A.jx, w, d);
  A.jy = sfma<cy>(A.jy, w, d);
  A.jz = sfma<cz>(A.jz, w, d);
  A.rxx = sfma<cx * cx>(A.rxx, w, s);
  A.ryy = sfma<cy * cy>(A.ryy, w, s);
  A.rzz = sfma<cz * cz>(A.rzz, w, s);
  A.rxy = sfma<cx * cy>(A.rxy, w, s);
  A.rxz = sfma<cx * cz>(A.rxz, w, s);
  A.ryz = sfma<cy * cz>(A.ryz, w, s);
}

// ---------------------------------------------------------------------------------------------
// Packed FP32 accumulation (FFMA2/FADD2: two FP32 lanes per instruction on sm_100 and later).
// The non-axial direction pairs are taken two at a time ("couples"), preferring two pairs with the
// same |c_x|, |c_y|, |c_z| so that both lanes feed the same moments; each moment keeps two partial
// sums (lane 0: first pair, lane 1: second pair) that are added once at the end.
template <class L>
struct Couples {
  __host__ __device__ static constexpr bool rep(int q) {  // one direction of each non-axial pair
    return q < L::opp(q) && !(L::cx(q) == 0 && L::cy(q) == 0);
  }
  __host__ __device__ static constexpr int support(int q) {
    return 4 * (L::cx(q) != 0) + 2 * (L::cy(q) != 0) + (L::cz(q) != 0);
  }
  __host__ __device__ static constexpr int count() {
    int n = 0;
    for (int q = 0; q < L::Q; ++q)
      if (rep(q)) ++n;
    return n / 2;
  }
  // first and second pair of couple k: greedy, same support first, then any
  __host__ __device__ static constexpr int member(int k, int which) {
    bool used[27] = {};
    for (int c = 0; c <= k; ++c) {
      int qa = -1, qb = -1;
      for (int q = 0; q < L::Q && qa < 0; ++q)
        if (rep(q) && !used[q]) qa = q;
      if (qa < 0) return -1;
      used[qa] = true;
      for (int q = 0; q < L::Q && qb < 0; ++q)
        if (rep(q) && !used[q] && support(q) == support(qa)) qb = q;
      for (int q = 0; q < L::Q && qb < 0; ++q)
        if (rep(q) && !used[q]) qb = q;
      if (qb < 0) return -1;
      used[qb] = true;
      if (c == k) return which == 0 ? qa : qb;
    }
    return -1;
  }
};

struct Accum2 {
  float2 a0, jx, jy, jz, rxx, ryy, rzz, rxy, rxz, ryz;
};

// acc + (CA wa, CB wb) v, elementwise, for compile-time CA, CB in {-1, 0, 1}
template <int CA, int CB>
__device__ __forceinline__ void pfma(float2& acc, float wa, float wb, float2 v) {
  if constexpr (CA != 0 || CB != 0) acc = __ffma2_rn(make_float2(float(CA) * wa, float(CB) * wb), v, acc);
}

// adds the two pairs of a couple: lane 0 (g.x, o.x) along qa and its opposite, lane 1 along qb
template <class L, int qa, int qb>
__device__ __forceinline__ void accumulate_couple(Accum2& A, float2 g, float2 o) {
  constexpr float wa = float(L::w(qa)), wb = float(L::w(qb));
  constexpr int ax = L::cx(qa), ay = L::cy(qa), az = L::cz(qa);
  constexpr int bx = L::cx(qb), by = L::cy(qb), bz = L::cz(qb);
  const float2 s = __fadd2_rn(g, o);
  const float2 d = __ffma2_rn(o, make_float2(-1.0f, -1.0f), g);
  A.a0 = __ffma2_rn(make_float2(wa, wb), s, A.a0);
  pfma<ax, bx>(A.jx, wa, wb, d);
  pfma<ay, by>(A.jy, wa, wb, d);
  pfma<az, bz>(A.jz, wa, wb, d);
  pfma<ax * ax, bx * bx>(A.rxx, wa, wb, s);
  pfma<ay * ay, by * by>(A.ryy, wa, wb, s);
  pfma<az * az, bz * bz>(A.rzz, wa, wb, s);
  pfma<ax * ay, bx * by>(A.rxy, wa, wb, s);
  pfma<ax * az, bx * bz>(A.rxz, wa, wb, s);
  pfma<ay * az, by * bz>(A.ryz, wa, wb, s);
}

#ifndef LBF_PACKED_ACC
#define LBF_PACKED_ACC 1
#endif

template <int BY>
struct FwdTile {
  static constexpr int ROWS = BY + 2;
  static constexpr int THREADS = 32 * ROWS;
  static constexpr int XOUT = 30;
};

// shared memory of a ring that keeps all Q populations of 3 planes (used by the adjoint kernel)
template <class L, class T, int BY, bool MASK>
constexpr size_t ring3_smem_bytes() {
  return size_t(3) * L::Q * FwdTile<BY>::ROWS * 32 * sizeof(T) + (MASK ? size_t(3) * FwdTile<BY>::ROWS * 32 : 0);
}

// ---------------------------------------------------------------------------------------------
// Population ring of the forward kernel, split by c_z. A population of plane p travelling along c
// is read by the output plane p + c_z, and (bounce-back) by its own site at plane p. With the two
// barriers of an iteration (after staging plane z+1, after the outputs of plane z) a group needs
//   c_z = -1: 2 plane slots, c_z = 0: 2 slots, c_z = +1: 3 slots.
// The three axial directions (rest, (0,0,+1), (0,0,-1)) only move along the thread's own column
// and live in registers, so the ring holds Q - 3 directions.
template <class L>
struct Dirs {
  __host__ __device__ static constexpr bool axial(int q) { return L::cx(q) == 0 && L::cy(q) == 0; }
  __host__ __device__ static constexpr int group(int q) { return L::cz(q) + 1; }
  __host__ __device__ static constexpr int gidx(int q) {
    int n = 0;
    for (int k = 0; k < q; ++k)
      if (!axial(k) && group(k) == group(q)) ++n;
    return n;
  }
  __host__ __device__ static constexpr int gsize(int g) {
    int n = 0;
    for (int k = 0; k < L::Q; ++k)
      if (!axial(k) && group(k) == g) ++n;
    return n;
  }
  __host__ __device__ static constexpr int find(int cx, int cy, int cz) {
    for (int k = 0; k < L::Q; ++k)
      if (L::cx(k) == cx && L::cy(k) == cy && L::cz(k) == cz) return k;
    return -1;
  }
};

// plane slots per group: c_z = -1 needs the plane being pulled (z+1) and, for bounce-back only,
// the own plane z; c_z = 0 the pulled plane z and the one being staged; c_z = +1 the pulled plane
// z-1, the plane z kept for the next output and the one being staged
template <class L, int ROWS, bool MASK = true>
struct GroupRing {
  using D = Dirs<L>;
  static constexpr int SITES = ROWS * 32;
  static constexpr int NS0 = MASK ? 2 : 1, NS1 = 2, NS2 = 3;
  __host__ __device__ static constexpr int base(int g) {
    return g == 0 ? 0 : (g == 1 ? NS0 * D::gsize(0) * SITES : (NS0 * D::gsize(0) + NS1 * D::gsize(1)) * SITES);
  }
  static constexpr int VALUES = (NS0 * D::gsize(0) + NS1 * D::gsize(1) + NS2 * D::gsize(2)) * SITES;
};

// TMA box of one plane patch: all 10 fields x ROWS rows x BX columns. The first column is the
// lane-0 site rounded down to a 16-byte boundary (A elements), so BX covers 32 lanes + A - 1.
template <class S>
struct TmaBox {
  static constexpr int A = 16 / int(sizeof(S));
  static constexpr int BX = ((32 + A - 1) + A - 1) / A * A;
};
// plane patches in flight per CTA (TMA stages)
#ifndef LBF_RAW_STAGES
#define LBF_RAW_STAGES 2
#endif
constexpr int kRawStages = LBF_RAW_STAGES;

// a TMA destination in shared memory must start on a 128-byte boundary: every stage of the raw
// ring is padded to a multiple of 128 bytes and the ring itself is aligned inside the dynamic
// shared memory (128 bytes of slack)
template <class S, int ROWS>
constexpr size_t raw_stage_bytes() {
  return (size_t(10) * ROWS * TmaBox<S>::BX * sizeof(S) + 127) / 128 * 128;
}

// elements (ring) / bytes (solid flags) of slack on each side; the edge lanes of an output row
// read at most 33 entries before or after their row
constexpr int kRingPad = 40;

template <class L, class S, int BY, bool MASK, bool TMA>
constexpr size_t fwd_smem_bytes() {
  using T = typename ComputeOf<S>::type;
  const size_t raw = TMA ? 128 + size_t(kRawStages) * raw_stage_bytes<S, BY + 2>() : 0;
  return raw + size_t(GroupRing<L, BY + 2, MASK>::VALUES + 2 * kRingPad) * sizeof(T) +
         (MASK ? size_t(3) * (BY + 2) * 32 + 2 * kRingPad : 0);
}

// per-site inputs other than the 10 stored fields, prefetched one plane ahead. TWO: 0 single
// component, 1 two components at equal densities, 2 two components with a density contrast
template <class T, int TWO>
struct SiteExtra {
  T F[3];     // force at the site: uniform (+ field), or F^n for two components
  T phi_o;    // two components: phi^n (source side)
  T Fn[3];    // two components: F^{n+1} (correction side; with a contrast F^s + F^b only)
  T phi_n;    // two components: phi^{n+1}
  T gphi[3];  // density contrast: grad phi^{n+1}
  bool solid;
};

// output rows per CTA and the minimum resident CTAs per SM asked of the register allocator, per
// lattice and storage width (bytes per stored value). D3Q19 FP32: 8 rows, 3 CTAs of 320 threads
// (<= 64 registers), limited by shared memory to 3. D3Q27: its larger ring fits 2 CTAs of 8 rows
// (<= 96 registers); with 16-bit storage the TMA stages are half as large and 6-row CTAs fit 3.
#ifndef LBF_FWD_ROWS_Q19
#define LBF_FWD_ROWS_Q19 8
#endif
#ifndef LBF_FWD_ROWS_Q27
#define LBF_FWD_ROWS_Q27 8
#endif
#ifndef LBF_FWD_ROWS_Q19_16
#define LBF_FWD_ROWS_Q19_16 8
#endif
#ifndef LBF_FWD_ROWS_Q27_16
#define LBF_FWD_ROWS_Q27_16 8
#endif
#ifndef LBF_FWD_ROWS_F64
#define LBF_FWD_ROWS_F64 4
#endif
#ifndef LBF_FWD_MINB_Q19
#define LBF_FWD_MINB_Q19 3
#endif
#ifndef LBF_FWD_MINB_Q27
#define LBF_FWD_MINB_Q27 2
#endif
#ifndef LBF_FWD_MINB_Q19_16
#define LBF_FWD_MINB_Q19_16 3
#endif
#ifndef LBF_FWD_MINB_Q27_16
#define LBF_FWD_MINB_Q27_16 2
#endif
// D3Q27 without walls: its ring needs one c_z = -1 slot less, and shorter tiles then fit 3 CTAs
// per SM (FP32: 6 rows, 72.6 KB; 16-bit: 7 rows, 70.3 KB; measured +4% over 8-row tiles at 2 CTAs)
#ifndef LBF_FWD_ROWS_Q27_NM
#define LBF_FWD_ROWS_Q27_NM 6
#endif
#ifndef LBF_FWD_MINB_Q27_NM
#define LBF_FWD_MINB_Q27_NM 3
#endif
#ifndef LBF_FWD_ROWS_Q27_16_NM
#define LBF_FWD_ROWS_Q27_16_NM 7
#endif
#ifndef LBF_FWD_MINB_Q27_16_NM
#define LBF_FWD_MINB_Q27_16_NM 3
#endif
// two-component D3Q19 FP32 (the droplet workload) has its own tile height: its per-site inputs
// (phase field, two force vectors) need more registers than the single-component kernel, and
// 7-row tiles (up to 72 registers at 3 CTAs/SM) remove the spills of 8-row ones (+2% at 128^3)
#ifndef LBF_FWD_ROWS_Q19_TWO
#define LBF_FWD_ROWS_Q19_TWO 7
#endif
#ifndef LBF_FWD_MINB_Q19_TWO
#define LBF_FWD_MINB_Q19_TWO 3
#endif
constexpr int fwd_rows(int Q, int bytes, bool mask = true, bool two = false) {
  if (two && Q == 19 && bytes == 4) return LBF_FWD_ROWS_Q19_TWO;
  return bytes == 8 ? LBF_FWD_ROWS_F64
                    : (bytes == 4 ? (Q == 19 ? LBF_FWD_ROWS_Q19 : (mask ? LBF_FWD_ROWS_Q27 : LBF_FWD_ROWS_Q27_NM))
                                  : (Q == 19 ? LBF_FWD_ROWS_Q19_16 : (mask ? LBF_FWD_ROWS_Q27_16 : LBF_FWD_ROWS_Q27_16_NM)));
}
// D3Q27h with 16-bit storage and no walls: 6-row tiles (up to 80 registers at 3 CTAs/SM), as
// the full-basis staging spills at the 72 registers of 7-row tiles
#ifndef LBF_FWD_ROWS_Q27H_16_NM
#define LBF_FWD_ROWS_Q27H_16_NM 6
#endif
constexpr int fwd_rows_lattice(int Q, int bytes, bool mask, bool two, bool high) {
  return (high && bytes == 2 && !mask) ? LBF_FWD_ROWS_Q27H_16_NM : fwd_rows(Q, bytes, mask, two);
}
constexpr int fwd_minb(int Q, int bytes, bool mask = true, bool two = false) {
  if (two && Q == 19 && bytes == 4) return LBF_FWD_MINB_Q19_TWO;
  return bytes == 8 ? 1
                    : (bytes == 4 ? (Q == 19 ? LBF_FWD_MINB_Q19 : (mask ? LBF_FWD_MINB_Q27 : LBF_FWD_MINB_Q27_NM))
                                  : (Q == 19 ? LBF_FWD_MINB_Q19_16 : (mask ? LBF_FWD_MINB_Q27_16 : LBF_FWD_MINB_Q27_16_NM)));
}

constexpr uint32_t kWaitPolls = 1u << 20;  // bound of every mbarrier wait

// LBF_DEBUG builds check every shared-memory and global index of the step against the buffer it
// addresses; a failed check sets bit 3 of the error flags (reported as LBF_EINTERNAL) and never
// traps. Release builds compile the checks away.
#ifdef LBF_DEBUG
#define LBF_CHECK(flags, cond)        \
  do {                                \
    if (!(cond)) atomicOr(flags, 8u); \
  } while (0)
#else
#define LBF_CHECK(flags, cond) \
  do {                         \
  } while (0)
#endif

template <class L, class S, int BY, bool MASK, int TWO, bool FF, bool TMA, bool RN>
__global__ void __launch_bounds__(FwdTile<BY>::THREADS, fwd_minb(L::Q, int(sizeof(S)), MASK, TWO != 0))
    k_stream_collide(const FwdParams a, const __grid_constant__ CUtensorMap tmap) {
  using T = typename ComputeOf<S>::type;
  using D = Dirs<L>;
  using R = GroupRing<L, BY + 2, MASK>;
  constexpr int Q = L::Q;
  constexpr int ROWS = BY + 2;
  constexpr int SITES = ROWS * 32;
  constexpr int QREST = D::find(0, 0, 0);
  constexpr int QUP = D::find(0, 0, 1);
  constexpr int QDN = D::find(0, 0, -1);
  constexpr int BX = TmaBox<S>::BX, AL = TmaBox<S>::A;
  constexpr int STAGE_ELEMS = 10 * ROWS * BX;                                  // one box
  constexpr int STAGE_STRIDE = int(raw_stage_bytes<S, ROWS>() / sizeof(S));   // padded stage
  constexpr size_t RAW_BYTES = TMA ? 128 + size_t(kRawStages) * raw_stage_bytes<S, ROWS>() : 0;
  constexpr int G0 = D::gsize(0) * SITES, G1 = D::gsize(1) * SITES, G2 = D::gsize(2) * SITES;
  constexpr int GS2 = D::gsize(2);  // three-slot offsets: ring g2 = slot * G2, solid flags g2 / GS2
  constexpr bool SITEF = TWO || FF;  // per-site force (else the uniform force of the parameters)
  static_assert(fwd_smem_bytes<L, S, BY, MASK, TMA>() >= 6 * 512 * sizeof(double), "smem too small for the final tree");
  static_assert(FwdTile<BY>::THREADS <= 512, "final tree assumes <= 512 threads");

  extern __shared__ __align__(128) unsigned char smem_raw[];
  S* rawst = reinterpret_cast<S*>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
  // population ring and solid-flag ring, each with kRingPad elements of slack on both sides: the
  // edge lanes of an output row read one element beyond their row (results discarded)
  T* ring = reinterpret_cast<T*>(smem_raw + RAW_BYTES) + kRingPad;
  uint8_t* msk = reinterpret_cast<uint8_t*>(ring + R::VALUES + kRingPad) + kRingPad;
  __shared__ __align__(8) uint64_t bars[kRawStages];
  __shared__ int abort_flag;

  const S* __restrict__ src = static_cast<const S*>(a.src);
  S* __restrict__ dst = static_cast<S*>(a.dst);
  const T* __restrict__ ffield = static_cast<const T*>(a.force_field);

  const int lane = threadIdx.x, row = threadIdx.y;
  const int x0 = blockIdx.x * FwdTile<BY>::XOUT;
  const int yb = a.y_begin, yrows = a.y_rows > 0 ? a.y_rows : a.ny;
  const int ty0 = yb + int(blockIdx.y) * BY;  // first output row of the tile (may exceed ny: wraps)
  const int gx = x0 - 1 + lane;
  const int gy = ty0 - 1 + row;
  const int ly = gy - yb;                     // row within this launch's range
  const int sx = ((gx % a.nx) + a.nx) % a.nx;
  const int sy = ((gy % a.ny) + a.ny) % a.ny;
  const bool out_row = row >= 1 && row <= BY;  // warp-uniform
  const bool outcol = out_row && lane >= 1 && lane <= FwdTile<BY>::XOUT && gx < a.nx && ly < yrows;
  const bool inbox = gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny;  // TMA delivers this site
  const bool needed = gx <= a.nx && ly <= yrows;                     // read by some output
  const int xa = ((x0 - 1 + AL) / AL - 1) * AL;                      // floor to AL; x0 - 1 >= -1
  const int xoff = x0 - 1 - xa;
  const long long plane = (long long)a.nx * a.ny;
  const int col = sy * a.nx + sx;
  const long long N = a.N;
  const int z0 = blockIdx.z * a.zchunk;
  const int z1 = min(a.nz, z0 + a.zchunk);
  const int me = row * 32 + lane;
  const T one_m_omega = T(1) - pick<T>(a.omega, a.omega_f);
  const T Fu0 = pick<T>(a.force[0], a.force_f[0]), Fu1 = pick<T>(a.force[1], a.force_f[1]),
          Fu2 = pick<T>(a.force[2], a.force_f[2]);
  // planes of the chunk window are numbered r = p - (z0 - 1) >= 0: raw stage and the two-slot ring
  // groups use r & 1, the three-slot group and the solid flags rotate through three slots
  const int pbase = z0 - 1;
  const S* raw_me = rawst + row * BX + lane + xoff;  // this thread's site in stage 0

  int issued = pbase - 1;  // last plane whose TMA load was issued (elected thread)
  auto issue = [&](int p) {  // elected thread only
    if (p > z1 || abort_flag) return;
    const int s = (p - pbase) % kRawStages;
    S* dstp = rawst + s * STAGE_STRIDE;
    if ((smem_u32(dstp) & 127u) != 0u) {  // never issue a copy the hardware would reject
      atomicOr(a.flags, 4u);
      abort_flag = 1;
      return;
    }
    // no proxy fence: the stage is only read through the generic proxy, and every read of it
    // completed before the barrier that precedes this call
    LBF_CHECK(a.flags, (xa * int(sizeof(S))) % 16 == 0 && s >= 0 && s < kRawStages);
    mbar_arrive_expect_tx(&bars[s], uint32_t(STAGE_ELEMS * sizeof(S)));
    tma_load_4d(dstp, &tmap, &bars[s], xa, ty0 - 1, wrap(p, a.nz), 0);
    issued = p;
  };
  auto wait_plane = [&](int p) {
    if (abort_flag) return;
    const int s = (p - pbase) % kRawStages;
    const uint32_t parity = uint32_t((p - pbase) / kRawStages) & 1u;
    if (!mbar_wait_bounded(&bars[s], parity, kWaitPolls)) {
      atomicOr(a.flags, 2u);
      abort_flag = 1;
    }
  };

  // -- per-site extras (mask, force, phase field), register prefetch ---------------------------
  auto load_extra = [&](int zp, SiteExtra<T, TWO>& e) {
    const long long zoff = (long long)wrap(zp, a.nz) * plane;
    if constexpr (TWO) {
      const T* po = static_cast<const T*>(a.phi_old) + zoff;
      const T* Fo = static_cast<const T*>(a.F_old) + zoff;
      e.phi_o = __ldg(po + col);
      e.F[0] = __ldg(Fo + col);
      e.F[1] = __ldg(Fo + N + col);
      e.F[2] = __ldg(Fo + 2 * N + col);
      if (outcol) {
        const T* pn = static_cast<const T*>(a.phi_new) + zoff;
        const T* Fn = static_cast<const T*>(a.F_new) + zoff;
        e.phi_n = __ldg(pn + col);
        // F_new is rewritten by this kernel only at the site's own output, after this read
        e.Fn[0] = Fn[col];
        e.Fn[1] = Fn[N + col];
        e.Fn[2] = Fn[2 * N + col];
        if constexpr (TWO == 2) {
          const T* gp = static_cast<const T*>(a.grad_phi) + zoff;
          e.gphi[0] = __ldg(gp + col);
          e.gphi[1] = __ldg(gp + N + col);
          e.gphi[2] = __ldg(gp + 2 * N + col);
        }
      }
    } else if constexpr (FF) {
      const T* fb = ffield + zoff;
      e.F[0] = Fu0 + __ldg(fb + col);
      e.F[1] = Fu1 + __ldg(fb + N + col);
      e.F[2] = Fu2 + __ldg(fb + 2 * N + col);
    }
    if constexpr (MASK) e.solid = __ldg(a.mask + zoff + col) != 0;
    else e.solid = false;
  };

  // the 10 stored values of this thread's site in plane p (raw stage `st` when staged by TMA).
  // With scaled 16-bit storage the six N fields are returned in storage units: N enters the
  // post-collision moments only through (1 - omega) N, so its power-of-two decode factor is applied
  // to (1 - omega) instead (exact, one multiply instead of six)
  auto read_raw = [&](int p, int st, T (&m)[10]) {
    if (TMA && inbox) {
      const S* b = raw_me + st * STAGE_STRIDE;
      LBF_CHECK(a.flags, st >= 0 && st < kRawStages && lane + xoff < BX &&
                             (b - rawst) + 9 * ROWS * BX < kRawStages * STAGE_STRIDE);
#pragma unroll
      for (int k = 0; k < 10; ++k) {
        const float dec = k == 0 ? a.sc.dec[0] : a.sc.dec[1];
        if constexpr (Codec<S>::scaled)
          m[k] = k < 4 ? static_cast<T>(static_cast<float>(b[k * ROWS * BX]) * dec)
                       : static_cast<T>(static_cast<float>(b[k * ROWS * BX]));
        else
          m[k] = static_cast<T>(b[k * ROWS * BX]);
      }
    } else if (needed || !TMA) {
      const S* __restrict__ bz = src + (long long)wrap(p, a.nz) * plane;
#pragma unroll
      for (int k = 0; k < 10; ++k) {
        const float dec = k == 0 ? a.sc.dec[0] : (k < 4 ? a.sc.dec[1] : 1.0f);
        m[k] = ld_field<S, T>(bz + k * N, col, dec);
      }
    } else {
#pragma unroll
      for (int k = 0; k < 10; ++k) m[k] = T(0);
    }
  };

  // own-site values of the planes being output (carried from staging)
  T Fown[3] = {Fu0, Fu1, Fu2}, Fnext[3] = {Fu0, Fu1, Fu2};
  // two components: 1/(2 rho) at equal densities, rho_l and rho_h - rho_l with a contrast, and
  // nu_l, nu_h - nu_l with the rate at nu_l
  const T i2r_two = TWO ? T(0.5) / pick<T>(a.rho_l, a.rho_l_f) : T(0.5);
  const T rho_l_two = pick<T>(a.rho_l, a.rho_l_f), drho_two = pick<T>(a.rho_h - a.rho_l, a.drho_f);
  const T nu_l_two = pick<T>(a.nu_l, a.nu_l_f), dnu_two = pick<T>(a.nu_h - a.nu_l, a.dnu_f);
  const T omm_two = T(1) - T(1) / (T(3) * nu_l_two + T(0.5));
  T phi_own = T(0), phi_next = T(0);
  T gphi_own[3] = {T(0), T(0), T(0)}, gphi_next[3] = {T(0), T(0), T(0)};
  // axial populations of the own column: up(z-1), up(z), dn(z), rest(z) and the new plane's
  T up_m1 = T(0), up_0 = T(0), dn_0 = T(0), rest_0 = T(0);
  T up_new = T(0), dn_new = T(0), rest_new = T(0);
  bool sol_m1 = false, sol_0 = false, sol_new = false;
  // three-slot ring offsets (elements of the c_z = +1 group, bytes of the solid flags) of the
  // planes z-1, z, z+1; they rotate by one slot per plane
  int g2m = 0, g20 = G2, g2p = 2 * G2;

  // -- staging: post-collision populations of plane p into the ring ----------------------------
  // par: (p - pbase) & 1 (compile time); g2: the three-slot offset of plane p. halo: 0 for the
  // output rows (every direction); +1 / -1 for the y-halo row below / above the tile, which is
  // pulled only along the directions with c_y = +1 / -1 and stages only those
  auto stage = [&](auto par_c, auto halo_c, int p, int g2, const SiteExtra<T, TWO>& e) -> bool {
    constexpr int par = decltype(par_c)::value;
    constexpr int H = decltype(halo_c)::value;
    T m[10];
    // raw stage of plane p: (p - pbase) mod kRawStages, the plane parity when there are two
    read_raw(p, kRawStages == 2 ? par : (p - pbase) % kRawStages, m);
    T inv2rho = T(0.5), omm = one_m_omega;
    if constexpr (TWO) {
      // the source side takes rho(phi^n) and nu(phi^n) = nu_l + phi (nu_h - nu_l): at equal
      // densities 1/(2 rho) is a constant, and the rate is a constant when the viscosities agree
      if constexpr (TWO == 2)
        inv2rho = T(0.5) / (rho_l_two + e.phi_o * drho_two);
      else
        inv2rho = i2r_two;
      if (dnu_two != T(0)) omm = T(1) - T(1) / (T(3) * (nu_l_two + e.phi_o * dnu_two) + T(0.5));
      else omm = omm_two;
      if (outcol) {
        phi_next = e.phi_n;
        Fnext[0] = e.Fn[0];
        Fnext[1] = e.Fn[1];
        Fnext[2] = e.Fn[2];
        if constexpr (TWO == 2) {
          gphi_next[0] = e.gphi[0];
          gphi_next[1] = e.gphi[1];
          gphi_next[2] = e.gphi[2];
        }
      }
    } else if constexpr (FF) {
      Fnext[0] = e.F[0];
      Fnext[1] = e.F[1];
      Fnext[2] = e.F[2];
    }
    const T Fs0 = SITEF ? e.F[0] : Fu0, Fs1 = SITEF ? e.F[1] : Fu1, Fs2 = SITEF ? e.F[2] : Fu2;
    if constexpr (Codec<S>::scaled) omm *= a.sc.dec[2];  // N is in storage units (read_raw)
    T* w0 = ring + R::base(0) + (R::NS0 == 2 ? par : 0) * G0 + me;
    T* w1 = ring + R::base(1) + par * G1 + me;
    T* w2 = ring + R::base(2) + g2 + me;
    auto put = [&](auto qc, T v) {
      constexpr int q = decltype(qc)::value;
      if constexpr (q == QUP) {
        up_new = v;
      } else if constexpr (q == QDN) {
        dn_new = v;
      } else {
        constexpr int g = D::group(q);
        T* b = g == 0 ? w0 : (g == 1 ? w1 : w2);
        LBF_CHECK(a.flags, (b + D::gidx(q) * SITES) - ring >= 0 && (b + D::gidx(q) * SITES) - ring < R::VALUES);
        b[D::gidx(q) * SITES] = v;
      }
    };
    if constexpr (L::HIGH) {
      const T uv[3] = {m[1], m[2], m[3]};
      const T hv[3] = {Fs0 * inv2rho, Fs1 * inv2rho, Fs2 * inv2rho};
      const T Nt[3][3] = {{m[4], m[7], m[8]}, {m[7], m[5], m[9]}, {m[8], m[9], m[6]}};
      T g[27];
      full_populations<T>(m[0], uv, hv, Nt, omm, g);
      static_for<Q>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        if constexpr (q == QREST) {
          if constexpr (H == 0) rest_new = g[q];
        } else if constexpr (H == 0 || L::cy(q) == H) {
          put(qc, g[q]);
        }
      });
    } else {
      const PostColl<T> P = post_collision<T>(m[0], m[1], m[2], m[3], m[4], m[5], m[6], m[7], m[8], m[9], Fs0, Fs1,
                                              Fs2, inv2rho, omm);
      static_for<Q>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        constexpr bool need_q = H == 0 || L::cy(q) == H, need_o = H == 0 || L::cy(L::opp(q)) == H;
        if constexpr (q == QREST) {
          if constexpr (H == 0) rest_new = P.q0;
        } else if constexpr (q < L::opp(q) && (need_q || need_o)) {
          T fq, fo;
          pop_pair<L, q, T>(P, fq, fo);
          if constexpr (need_q) put(qc, fq);
          if constexpr (need_o) put(std::integral_constant<int, L::opp(q)>{}, fo);
        }
      });
    }
    if constexpr (MASK) msk[g2 / GS2 + me] = e.solid ? 1 : 0;
    sol_new = e.solid;
    return e.solid;
  };

  // the reduced halo staging pays on D3Q27 (9 of 26 directions per halo row); on D3Q19 (5 of 18)
  // the extra code measured slower than staging every direction
  auto stage_row = [&](auto par_c, int p, int g2, const SiteExtra<T, TWO>& e) -> bool {
    if constexpr (L::Q == 27 && !L::HIGH) {  // D3Q27h: one staging body (compile time)
      if (row == 0) return stage(par_c, std::integral_constant<int, 1>{}, p, g2, e);
      if (row == ROWS - 1) return stage(par_c, std::integral_constant<int, -1>{}, p, g2, e);
    }
    return stage(par_c, std::integral_constant<int, 0>{}, p, g2, e);
  };

  T red[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
  SiteExtra<T, TWO> ex;

  if (me == 0) {
    abort_flag = 0;
    if constexpr (TMA) {
      for (int s = 0; s < kRawStages; ++s) mbar_init(&bars[s], 1);
      fence_mbar_init();
    }
  }
  if constexpr (MASK) {
    // solid-flag padding read by the edge lanes: keep it defined
    for (int i = me; i < kRingPad; i += FwdTile<BY>::THREADS) {
      msk[-kRingPad + i] = 0;
      msk[3 * SITES + i] = 0;
    }
  }
  __syncthreads();
  if constexpr (TMA) {
    if (me == 0) {
      prefetch_tensormap(&tmap);
      for (int p = pbase; p < pbase + kRawStages; ++p) issue(p);
    }
  }

  // prologue: stage planes z0-1 (r = 0) and z0 (r = 1)
  load_extra(z0 - 1, ex);
  if constexpr (TMA) {
    wait_plane(z0 - 1);
  }
  bool any_m = stage_row(std::integral_constant<int, 0>{}, z0 - 1, g2m, ex);
  up_m1 = up_new;
  sol_m1 = sol_new;
  load_extra(z0, ex);
  if constexpr (MASK)
    any_m = __syncthreads_or(any_m);
  else
    __syncthreads();
  if constexpr (TMA) {
    if (me == 0) issue(z0 - 1 + kRawStages);
    wait_plane(z0);
  }
  bool any_0 = stage_row(std::integral_constant<int, 1>{}, z0, g20, ex);
  if constexpr (TMA) {
    if (!out_row) wait_plane(z0 + 1);  // staged by the first iteration (z0 + 1 <= z1)
  }
  up_0 = up_new;
  dn_0 = dn_new;
  rest_0 = rest_new;
  sol_0 = sol_new;
  Fown[0] = Fnext[0];
  Fown[1] = Fnext[1];
  Fown[2] = Fnext[2];
  phi_own = phi_next;
  gphi_own[0] = gphi_next[0];
  gphi_own[1] = gphi_next[1];
  gphi_own[2] = gphi_next[2];
  load_extra(z0 + 1, ex);
  if constexpr (MASK)
    any_0 = __syncthreads_or(any_0);
  else
    __syncthreads();
  if constexpr (TMA) {
    if (me == 0) issue(z0 + kRawStages);
  }

  // one plane: stage z+1, outputs of z. PAR = (z - z0) & 1 at compile time
  auto iteration = [&](auto par_c, int z) {
    constexpr int PAR = decltype(par_c)::value;
    // plane z+1 has landed: the y-halo warps waited for it before the barrier that ended the
    // previous iteration (or the prologue), and that barrier orders the observation for everyone
    bool any_p = stage_row(std::integral_constant<int, PAR>{}, z + 1, g2p, ex);
    load_extra(z + 2, ex);  // in flight during the outputs of plane z (z + 2 <= nz + 1 wraps)
    if constexpr (MASK)
      any_p = __syncthreads_or(any_p);
    else
      __syncthreads();
    if constexpr (TMA) {
      if (me == 0) issue(z + 1 + kRawStages);  // the stage of plane z+1 was consumed by everyone
    }
    if (out_row) {
      // pull bases: group c_z = -1 from plane z+1, c_z = 0 from plane z, c_z = +1 from plane z-1
      const T* P0 = ring + R::base(0) + (R::NS0 == 2 ? PAR : 0) * G0 + me;
      const T* P1 = ring + R::base(1) + (PAR ^ 1) * G1 + me;
      const T* P2 = ring + R::base(2) + g2m + me;
      auto gather = [&](auto walls_c) {
        constexpr bool W = decltype(walls_c)::value;
        const T* O0 = ring + R::base(0) + (R::NS0 == 2 ? (PAR ^ 1) : 0) * G0 + me;  // own site, plane z (walls only)
        const T* O2 = ring + R::base(2) + g20 + me;
        const uint8_t* MM = msk + g2m / GS2 + me;
        const uint8_t* M0 = msk + g20 / GS2 + me;
        const uint8_t* MP = msk + g2p / GS2 + me;
        Accum<T> A = {T(L::w(QREST)) * rest_0, T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
        auto pulled = [&](auto qc) -> T {
          constexpr int q = decltype(qc)::value;
          constexpr int cx = L::cx(q), cy = L::cy(q), cz = L::cz(q);
          constexpr int g = D::group(q);
          constexpr int off = D::gidx(q) * SITES - cy * 32 - cx;
          LBF_CHECK(a.flags, ((g == 0 ? P0 : (g == 1 ? P1 : P2)) + off) - ring >= -kRingPad &&
                                 ((g == 0 ? P0 : (g == 1 ? P1 : P2)) + off) - ring < R::VALUES + kRingPad);
          T v = (g == 0 ? P0 : (g == 1 ? P1 : P2))[off];
          if constexpr (W) {
            const uint8_t* mk = cz > 0 ? MM : (cz < 0 ? MP : M0);
            LBF_CHECK(a.flags, (mk - cy * 32 - cx) - msk >= -kRingPad && (mk - cy * 32 - cx) - msk < 3 * SITES + kRingPad);
            if (mk[-cy * 32 - cx]) {  // halfway bounce-back: own post-collision population of opp(q)
              constexpr int o = L::opp(q);
              constexpr int go = D::group(o);
              v = (go == 0 ? O0 : (go == 1 ? P1 : O2))[D::gidx(o) * SITES];
            }
          }
          return v;
        };
        if constexpr (std::is_same<T, float>::value && L::Q == 27 && LBF_PACKED_ACC) {
          using C = Couples<L>;
          const float2 z2 = make_float2(0.0f, 0.0f);
          Accum2 A2 = {z2, z2, z2, z2, z2, z2, z2, z2, z2, z2};
          static_for<C::count()>([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            constexpr int qa = C::member(k, 0), qb = C::member(k, 1);
            static_assert(qa >= 0 && qb >= 0, "direction couples");
            const float2 g = make_float2(pulled(std::integral_constant<int, qa>{}), pulled(std::integral_constant<int, qb>{}));
            const float2 o = make_float2(pulled(std::integral_constant<int, L::opp(qa)>{}),
                                         pulled(std::integral_constant<int, L::opp(qb)>{}));
            accumulate_couple<L, qa, qb>(A2, g, o);
          });
          A.a0 += A2.a0.x + A2.a0.y;
          A.jx = A2.jx.x + A2.jx.y;
          A.jy = A2.jy.x + A2.jy.y;
          A.jz = A2.jz.x + A2.jz.y;
          A.rxx = A2.rxx.x + A2.rxx.y;
          A.ryy = A2.ryy.x + A2.ryy.y;
          A.rzz = A2.rzz.x + A2.rzz.y;
          A.rxy = A2.rxy.x + A2.rxy.y;
          A.rxz = A2.rxz.x + A2.rxz.y;
          A.ryz = A2.ryz.x + A2.ryz.y;
        } else {
          static_for<Q>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            if constexpr (q != QREST && q < L::opp(q) && q != QUP && q != QDN) {
              const T fq = pulled(qc);
              const T fo = pulled(std::integral_constant<int, L::opp(q)>{});
              accumulate_pair<L::cx(q), L::cy(q), L::cz(q), T>(A, fq, fo, T(L::w(q)));
            }
          });
        }
        // axial pair: (0,0,+1) comes from the plane below, (0,0,-1) from the plane above
        T fup = up_m1, fdn = dn_new;
        if constexpr (W) {
          if (sol_m1) fup = dn_0;
          if (sol_new) fdn = up_0;
        }
        accumulate_pair<0, 0, 1, T>(A, fup, fdn, T(L::w(QUP)));
        return A;
      };
      Accum<T> A;
      if constexpr (MASK) {
        if (any_m || any_0 || any_p)
          A = gather(std::true_type{});
        else
          A = gather(std::false_type{});
      } else {
        A = gather(std::false_type{});
      }
      // Eq. (corr): u = a1 + F/(2 rho), a2 = (sum c c f - cs2 a0 delta) + (u F + F u)/(2 rho)
      T i2r = i2r_two;
      if constexpr (TWO == 2) {
        // density contrast (Sec. 2 force split): the force of the new state adds to F^s + F^b
        //   F^p = -p* cs2 grad rho and F^nu = -(nu omega / cs2) a*_neq . grad rho,
        // with p* = a*0 and a*_neq = a*2 - a*1 a*1 the raw moments just streamed in (the
        // uncorrected a*1), rho, nu, omega and grad rho = (rho_h - rho_l) grad phi at phi^{n+1}
        const T rho_n = rho_l_two + phi_own * drho_two;
        i2r = T(0.5) / rho_n;
        const T gr0 = drho_two * gphi_own[0], gr1 = drho_two * gphi_own[1], gr2 = drho_two * gphi_own[2];
        const T p3 = A.a0 * (T(1) / T(3));
        const T qxx = (A.rxx - p3) - A.jx * A.jx, qyy = (A.ryy - p3) - A.jy * A.jy, qzz = (A.rzz - p3) - A.jz * A.jz;
        const T qxy = A.rxy - A.jx * A.jy, qxz = A.rxz - A.jx * A.jz, qyz = A.ryz - A.jy * A.jz;
        const T nu_n = nu_l_two + phi_own * dnu_two;
        const T cnu = T(-3) * nu_n / (T(3) * nu_n + T(0.5));
        Fown[0] += -p3 * gr0 + cnu * (qxx * gr0 + qxy * gr1 + qxz * gr2);
        Fown[1] += -p3 * gr1 + cnu * (qxy * gr0 + qyy * gr1 + qyz * gr2);
        Fown[2] += -p3 * gr2 + cnu * (qxz * gr0 + qyz * gr1 + qzz * gr2);
        if (outcol && !sol_0) {
          T* Fw = static_cast<T*>(a.F_new) + (long long)z * plane + col;
          Fw[0] = Fown[0];
          Fw[N] = Fown[1];
          Fw[2 * N] = Fown[2];
        }
      }
      const T hx = (SITEF ? Fown[0] : Fu0) * i2r, hy = (SITEF ? Fown[1] : Fu1) * i2r,
              hz = (SITEF ? Fown[2] : Fu2) * i2r;
      const T ux = A.jx + hx, uy = A.jy + hy, uz = A.jz + hz;
      const T a0c = A.a0 * (T(1) / T(3));
      const T nxx = (A.rxx - a0c) + T(2) * ux * hx - ux * ux;
      const T nyy = (A.ryy - a0c) + T(2) * uy * hy - uy * uy;
      const T nzz = (A.rzz - a0c) + T(2) * uz * hz - uz * uz;
      const T nxy = A.rxy + (ux * hy + hx * uy) - ux * uy;
      const T nxz = A.rxz + (ux * hz + hx * uz) - ux * uz;
      const T nyz = A.ryz + (uy * hz + hy * uz) - uy * uz;
      const T uu = ux * ux + uy * uy + uz * uz;
      if (outcol && !sol_0) {
        const long long zc = (long long)z * plane + col;
        LBF_CHECK(a.flags, z >= 0 && z < a.nz && col >= 0 && col < plane && zc + 9 * N < 10 * N);
        // random sequence of this site and step (16-bit storage only)
        {
          // 16-bit storage rounds p* and u stochastically unless RN (round to nearest); the six N
          // fields always round to nearest: N is recomputed from the populations every step rather
          // than accumulated, so its small changes are never lost (stochastic rounding of N gave the
          // same error at 64^3 and 512^3 and costs two instructions per field). FP32/FP64 stores
          // are plain.
          uint32_t rs = Codec<S>::scaled && !RN ? fmix32(uint32_t(zc) ^ a.salt) : 0u;
          st_field<S, RN>(dst, zc, A.a0, a.sc.enc[0], rs);
          st_field<S, RN>(dst + N, zc, ux, a.sc.enc[1], rs);
          st_field<S, RN>(dst + 2 * N, zc, uy, a.sc.enc[1], rs);
          st_field<S, RN>(dst + 3 * N, zc, uz, a.sc.enc[1], rs);
          st_field<S, true>(dst + 4 * N, zc, nxx, a.sc.enc[2], rs);
          st_field<S, true>(dst + 5 * N, zc, nyy, a.sc.enc[2], rs);
          st_field<S, true>(dst + 6 * N, zc, nzz, a.sc.enc[2], rs);
          st_field<S, true>(dst + 7 * N, zc, nxy, a.sc.enc[2], rs);
          st_field<S, true>(dst + 8 * N, zc, nxz, a.sc.enc[2], rs);
          st_field<S, true>(dst + 9 * N, zc, nyz, a.sc.enc[2], rs);
        }
        if (!(uu <= T(a.umax2))) atomicOr(a.flags, 1u);
        red[0] += A.a0;
        red[1] += ux;
        red[2] += uy;
        red[3] += uz;
        if constexpr (TWO) red[4] += phi_own;
        red[5] += uu;
      }
    }
    // rotate the own-column carries and the three-slot offsets to plane z+1
    up_m1 = up_0;
    up_0 = up_new;
    dn_0 = dn_new;
    rest_0 = rest_new;
    sol_m1 = sol_0;
    sol_0 = sol_new;
    Fown[0] = Fnext[0];
    Fown[1] = Fnext[1];
    Fown[2] = Fnext[2];
    phi_own = phi_next;
    gphi_own[0] = gphi_next[0];
    gphi_own[1] = gphi_next[1];
    gphi_own[2] = gphi_next[2];
    any_m = any_0;
    any_0 = any_p;
    const int g2t = g2m;
    g2m = g20;
    g20 = g2p;
    g2p = g2t;
    if constexpr (TMA) {
      if (!out_row && z + 2 <= z1) wait_plane(z + 2);  // staged by the next iteration
    }
    __syncthreads();
  };

  for (int z = z0; z < z1 && !abort_flag; z += 2) {
    iteration(std::integral_constant<int, 0>{}, z);
    if (z + 1 < z1 && !abort_flag) iteration(std::integral_constant<int, 1>{}, z + 1);
  }

  if constexpr (TMA) {
    // after an aborted wait, let the copies still in flight land before the CTA exits (bounded)
    if (abort_flag && me == 0) {
      for (int p = max(pbase, issued - kRawStages + 1); p <= issued; ++p) {
        const int s = (p - pbase) % kRawStages;
        mbar_wait_bounded(&bars[s], uint32_t((p - pbase) / kRawStages) & 1u, kWaitPolls);
      }
    }
  }

  if (a.partials != nullptr) {
    // warp sums in the compute type, block and grid sums in FP64 (scratch: the idle ring)
    double* red_s = reinterpret_cast<double*>(smem_raw + RAW_BYTES);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      T v = red[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red_s[row * 6 + k] = static_cast<double>(v);
    }
    __syncthreads();
    const long long nb = (long long)gridDim.x * gridDim.y * gridDim.z;
    if (me < 6) {
      double s = 0.0;
      for (int r = 0; r < ROWS; ++r) s += red_s[r * 6 + me];
      const long long b = a.block_base + ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
      a.partials[b * 8 + me] = s;
    }
    // second stage in the same launch: the last block to finish sums the partials in a fixed
    // order (thread t takes blocks t, t + T, ...; then a fixed tree), so the result is
    // deterministic and a step is a single kernel
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    const long long nall = a.final_blocks > 0 ? a.final_blocks : a.block_base + nb;  // partials to add
    if (me == 0) last = atomicAdd(a.counter, 1u) == (unsigned)(a.final_blocks > 0 ? nall - 1 : nb - 1);
    __syncthreads();
    if (last) {
      __threadfence();
      constexpr int NT = FwdTile<BY>::THREADS;
      double* tree = reinterpret_cast<double*>(smem_raw);
      for (int i = me; i < 6 * 512; i += NT) tree[i] = 0.0;
      __syncthreads();
      for (int k = 0; k < 6; ++k) {
        double acc = 0.0;
        for (long long b = me; b < nall; b += NT) acc += __ldcg(a.partials + b * 8 + k);
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
