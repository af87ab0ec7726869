// Fused pull-stream-and-collide step with two sites per thread (FP32 storage, single component).
//
// Same method, tile and plane march as k_stream_collide (stream_collide.cuh; Sec. 2, Eq. (pullLLB)
// followed by Eq. (corr)): a CTA owns 30 x BY output sites of an x-y tile, loads each plane of
// its patch with one TMA box, stages the post-collision populations of every site into a ring
// split by c_z and pulls them from planes z-1, z, z+1. What differs is the thread mapping:
//   * a thread owns the two sites of one column in the adjacent tile rows 2k and 2k+1, so a CTA of
//     (BY+2)/2 warps covers the BY output rows and the two y-halo rows with no idle warp;
//   * every arithmetic step runs on both sites at once with the packed FP32 instructions of
//     sm_100 and later (fma/add/sub/mul .f32x2: two FP32 lanes per instruction), which halves
//     the arithmetic issue slots per site;
//   * the ring interleaves the two rows of a pair (site (lane, r) at ((r / 2) * 32 + lane) * 2 +
//     r % 2), so both populations of a direction are stored with one 64-bit shared store and
//     pulled along c_y = 0 with one 64-bit load (two 32-bit loads along c_y = +/-1).
// The halo row of the first and last pair is evaluated with its partner and discarded; the
// arithmetic of a pair is the same for every site, so nothing diverges.
#pragma once

#include "stream_collide.cuh"

namespace lbf {

// -- packed FP32 pairs -------------------------------------------------------------------------
__device__ __forceinline__ float2 f2c(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  unsigned long long ra, rb, r;
  memcpy(&ra, &a, 8);
  memcpy(&rb, &b, 8);
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(ra), "l"(rb));
  float2 v;
  memcpy(&v, &r, 8);
  return v;
}
// acc + C v for a compile-time C in {-1, 0, 1}
template <int C>
__device__ __forceinline__ float2 sadd2(float2 acc, float2 v) {
  if constexpr (C > 0)
    return add2(acc, v);
  else if constexpr (C < 0)
    return sub2(acc, v);
  else
    return acc;
}
// acc + C w v for a compile-time C in {-1, 0, 1}
template <int C>
__device__ __forceinline__ float2 sfma2(float2 acc, float w, float2 v) {
  if constexpr (C != 0)
    return fma2(f2c(float(C) * w), v, acc);
  else
    return acc;
}

// post_collision of stream_collide.cuh for two sites; m = (p*, u, N) of both, h = F / (2 rho)
struct PostColl2 {
  float2 q0, bx, by, bz, exx, eyy, ezz, exy, exz, eyz;
};

__device__ __forceinline__ PostColl2 post_collision2(const float2 (&m)[10], float2 hx, float2 hy, float2 hz,
                                                     float2 omm) {
  const float2 ux = m[1], uy = m[2], uz = m[3];
  const float2 two = f2c(2.0f);
  // P_aa = u_a (u_a + 2 h_a) + (1 - omega) N_aa,  P_ab = u_a (u_b + h_b) + h_a u_b + (1 - omega) N_ab
  const float2 pxx = fma2(ux, fma2(two, hx, ux), mul2(omm, m[4]));
  const float2 pyy = fma2(uy, fma2(two, hy, uy), mul2(omm, m[5]));
  const float2 pzz = fma2(uz, fma2(two, hz, uz), mul2(omm, m[6]));
  const float2 pxy = fma2(ux, add2(uy, hy), fma2(hx, uy, mul2(omm, m[7])));
  const float2 pxz = fma2(ux, add2(uz, hz), fma2(hx, uz, mul2(omm, m[8])));
  const float2 pyz = fma2(uy, add2(uz, hz), fma2(hy, uz, mul2(omm, m[9])));
  PostColl2 r;
  r.q0 = fma2(f2c(-1.5f), add2(add2(pxx, pyy), pzz), m[0]);
  const float2 three = f2c(3.0f);
  r.bx = mul2(three, add2(ux, hx));
  r.by = mul2(three, add2(uy, hy));
  r.bz = mul2(three, add2(uz, hz));
  const float2 c45 = f2c(4.5f), c9 = f2c(9.0f);
  r.exx = mul2(c45, pxx);
  r.eyy = mul2(c45, pyy);
  r.ezz = mul2(c45, pzz);
  r.exy = mul2(c9, pxy);
  r.exz = mul2(c9, pxz);
  r.eyz = mul2(c9, pyz);
  return r;
}

// pop_pair of stream_collide.cuh for two sites: f_q / w_q = s + d and f_opp(q) / w_q = s - d with
// s = q0 + c.e.c and d = c.b; d is formed with its leading component positive and the sign of
// that component decides which of s +/- d is f_q
template <class L, int q>
__device__ __forceinline__ void pop_pair2(const PostColl2& P, float2& fq, float2& fo) {
  constexpr int cx = L::cx(q), cy = L::cy(q), cz = L::cz(q);
  float2 s = P.q0;
  s = sadd2<cx * cx>(s, P.exx);
  s = sadd2<cy * cy>(s, P.eyy);
  s = sadd2<cz * cz>(s, P.ezz);
  s = sadd2<cx * cy>(s, P.exy);
  s = sadd2<cx * cz>(s, P.exz);
  s = sadd2<cy * cz>(s, P.eyz);
  constexpr int lead = cx != 0 ? cx : (cy != 0 ? cy : cz);  // +1 or -1
  float2 d;
  if constexpr (cx != 0) {
    d = sadd2<cz * lead>(sadd2<cy * lead>(P.bx, P.by), P.bz);
  } else if constexpr (cy != 0) {
    d = sadd2<cz * lead>(P.by, P.bz);
  } else {
    d = P.bz;
  }
  if constexpr (lead > 0) {
    fq = add2(s, d);
    fo = sub2(s, d);
  } else {
    fq = sub2(s, d);
    fo = add2(s, d);
  }
}

struct Accum2S {
  float2 a0, jx, jy, jz, rxx, ryy, rzz, rxy, rxz, ryz;
};

// accumulate_pair of stream_collide.cuh for two sites
template <int cx, int cy, int cz>
__device__ __forceinline__ void accumulate_pair2(Accum2S& A, float2 gq, float2 go, float w) {
  const float2 s = add2(gq, go), d = sub2(gq, go);
  A.a0 = fma2(f2c(w), s, A.a0);
  A.jx = sfma2<cx>(A.jx, w, d);
  A.jy = sfma2<cy>(A.jy, w, d);
  A.jz = sfma2<cz>(A.jz, w, d);
  A.rxx = sfma2<cx * cx>(A.rxx, w, s);
  A.ryy = sfma2<cy * cy>(A.ryy, w, s);
  A.rzz = sfma2<cz * cz>(A.rzz, w, s);
  A.rxy = sfma2<cx * cy>(A.rxy, w, s);
  A.rxz = sfma2<cx * cz>(A.rxz, w, s);
  A.ryz = sfma2<cy * cz>(A.ryz, w, s);
}

// -- tile and shared memory ----------------------------------------------------------------------
template <int BY>
struct P2Tile {
  static_assert(BY % 2 == 0, "the rows of a tile (BY + 2) form pairs");
  static constexpr int ROWS = BY + 2;
  static constexpr int PAIRS = ROWS / 2;  // warps per CTA
  static constexpr int THREADS = 32 * PAIRS;
  static constexpr int XOUT = 30;
};

// output rows per CTA: D3Q19 8 (5 warps), D3Q27 6 (4 warps); both fit 3 CTAs per SM
#ifndef LBF_P2_ROWS_Q19
#define LBF_P2_ROWS_Q19 8
#endif
#ifndef LBF_P2_ROWS_Q27
#define LBF_P2_ROWS_Q27 6
#endif
#ifndef LBF_P2_MINB
#define LBF_P2_MINB 3
#endif
constexpr int p2_rows(int Q) { return Q == 19 ? LBF_P2_ROWS_Q19 : LBF_P2_ROWS_Q27; }

// A halo site of the first or last pair pulls from the row beyond the tile, at most 2 * 32 + 2 + 1
// values before its slot or 2 * 32 values after it; its result is discarded. Shared memory after
// the TMA stages: [solid flags, 3 x ROWS x 32 bytes | or kP2Pad zeros] [ring] [kP2Pad zeros]. The
// ring's front slack is the flag ring (bytes 0/1 read as floats are zero or subnormal) or zeros,
// so every value a discarded site reads is finite; the flag ring's own slack is the end of the
// TMA stages in front of it and the ring behind it (flags of discarded sites only).
constexpr int kP2Pad = 66;

template <class L, int BY, bool MASK>
constexpr size_t p2_front_bytes() {
  return MASK ? size_t(3) * (BY + 2) * 32 : size_t(kP2Pad) * sizeof(float);
}

template <class L, int BY, bool MASK>
constexpr size_t p2_smem_bytes() {
  return 128 + size_t(kRawStages) * raw_stage_bytes<float, BY + 2>() + p2_front_bytes<L, BY, MASK>() +
         size_t(GroupRing<L, BY + 2, MASK>::VALUES + kP2Pad) * sizeof(float);
}

// -- the kernel ----------------------------------------------------------------------------------
template <class L, int BY, bool MASK>
__global__ void __launch_bounds__(P2Tile<BY>::THREADS, LBF_P2_MINB)
    k_stream_collide_p2(const FwdParams a, const __grid_constant__ CUtensorMap tmap) {
  static_assert(!L::HIGH, "second-order Hermite truncation only");
  using D = Dirs<L>;
  using R = GroupRing<L, BY + 2, MASK>;
  constexpr int Q = L::Q;
  constexpr int ROWS = BY + 2;
  constexpr int SITES = ROWS * 32;
  constexpr int QREST = D::find(0, 0, 0);
  constexpr int QUP = D::find(0, 0, 1);
  constexpr int QDN = D::find(0, 0, -1);
  constexpr int BX = TmaBox<float>::BX, AL = TmaBox<float>::A;
  constexpr int STAGE_ELEMS = 10 * ROWS * BX;
  constexpr int STAGE_STRIDE = int(raw_stage_bytes<float, ROWS>() / sizeof(float));
  constexpr size_t RAW_BYTES = 128 + size_t(kRawStages) * raw_stage_bytes<float, ROWS>();
  constexpr int G0 = D::gsize(0) * SITES, G1 = D::gsize(1) * SITES, G2 = D::gsize(2) * SITES;
  constexpr int GS2 = D::gsize(2);
  constexpr int NT = P2Tile<BY>::THREADS;
  static_assert(p2_smem_bytes<L, BY, MASK>() >= 6 * 512 * sizeof(double), "smem too small for the final tree");
  static_assert(NT <= 512, "final tree assumes <= 512 threads");
  static_assert(SITES % 2 == 0, "64-bit ring accesses");

  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* rawst = reinterpret_cast<float*>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
  uint8_t* msk = smem_raw + RAW_BYTES;  // MASK only
  float* ring = reinterpret_cast<float*>(smem_raw + RAW_BYTES + p2_front_bytes<L, BY, MASK>());
  constexpr int FRONT = int(p2_front_bytes<L, BY, MASK>() / sizeof(float));  // readable values before the ring
  static_assert(FRONT >= kP2Pad && (RAW_BYTES + p2_front_bytes<L, BY, MASK>()) % 8 == 0, "ring slack");
  __shared__ __align__(8) uint64_t bars[kRawStages];
  __shared__ int abort_flag;

  const float* __restrict__ src = static_cast<const float*>(a.src);
  float* __restrict__ dst = static_cast<float*>(a.dst);

  const int lane = threadIdx.x, kp = threadIdx.y;  // kp: row pair (tile rows 2 kp, 2 kp + 1)
  const int me = kp * 32 + lane;
  const int ob = me * 2;  // ring index of this thread's pair
  const int x0 = blockIdx.x * P2Tile<BY>::XOUT;
  const int gx = x0 - 1 + lane;
  const int gy0 = int(blockIdx.y) * BY - 1 + 2 * kp, gy1 = gy0 + 1;
  const int sx = ((gx % a.nx) + a.nx) % a.nx;
  const int sy0 = ((gy0 % a.ny) + a.ny) % a.ny, sy1 = ((gy1 % a.ny) + a.ny) % a.ny;
  const bool lane_out = lane >= 1 && lane <= P2Tile<BY>::XOUT && gx < a.nx;
  const bool out0 = lane_out && 2 * kp >= 1 && gy0 < a.ny;        // row 2 kp <= BY always
  const bool out1 = lane_out && 2 * kp + 1 <= BY && gy1 < a.ny;   // row 2 kp + 1 >= 1 always
  const bool xin = gx >= 0 && gx < a.nx;
  const bool inbox0 = xin && gy0 >= 0 && gy0 < a.ny, inbox1 = xin && gy1 >= 0 && gy1 < a.ny;  // TMA delivers
  const bool need0 = gx <= a.nx && gy0 <= a.ny, need1 = gx <= a.nx && gy1 <= a.ny;           // read by an output
  const int xa = ((x0 - 1 + AL) / AL - 1) * AL;  // floor to AL; x0 - 1 >= -1
  const int xoff = x0 - 1 - xa;
  const long long plane = (long long)a.nx * a.ny;
  const int col0 = sy0 * a.nx + sx, col1 = sy1 * a.nx + sx;
  const long long N = a.N;
  const int z0 = blockIdx.z * a.zchunk;
  const int z1 = min(a.nz, z0 + a.zchunk);
  const float2 omm2 = f2c(1.0f - a.omega_f);
  // uniform force: h = F / (2 rho) with rho = 1
  const float2 hx2 = f2c(0.5f * a.force_f[0]), hy2 = f2c(0.5f * a.force_f[1]), hz2 = f2c(0.5f * a.force_f[2]);
  const float2 tx2 = f2c(a.force_f[0]), ty2 = f2c(a.force_f[1]), tz2 = f2c(a.force_f[2]);  // 2 h
  const int pbase = z0 - 1;
  const float* raw_me = rawst + (2 * kp) * BX + lane + xoff;  // site of row 2 kp in stage 0

  int issued = pbase - 1;
  auto issue = [&](int p) {  // thread 0 only
    if (p > z1 || abort_flag) return;
    const int s = (p - pbase) % kRawStages;
    float* dstp = rawst + s * STAGE_STRIDE;
    if ((smem_u32(dstp) & 127u) != 0u) {
      atomicOr(a.flags, 4u);
      abort_flag = 1;
      return;
    }
    LBF_CHECK(a.flags, (xa * int(sizeof(float))) % 16 == 0 && s >= 0 && s < kRawStages);
    mbar_arrive_expect_tx(&bars[s], uint32_t(STAGE_ELEMS * sizeof(float)));
    tma_load_4d(dstp, &tmap, &bars[s], xa, int(blockIdx.y) * BY - 1, wrap(p, a.nz), 0);
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

  // the 10 stored values of both sites in plane p (raw stage st)
  auto read_raw = [&](int p, int st, float2 (&m)[10]) {
    const float* b = raw_me + st * STAGE_STRIDE;
    const float* bz = src + (long long)wrap(p, a.nz) * plane;
    LBF_CHECK(a.flags, st >= 0 && st < kRawStages && lane + xoff < BX &&
                           (b - rawst) + BX + 9 * ROWS * BX < kRawStages * STAGE_STRIDE);
#pragma unroll
    for (int f = 0; f < 10; ++f) {
      m[f].x = inbox0 ? b[f * ROWS * BX] : (need0 ? __ldg(bz + f * N + col0) : 0.0f);
      m[f].y = inbox1 ? b[f * ROWS * BX + BX] : (need1 ? __ldg(bz + f * N + col1) : 0.0f);
    }
  };

  // axial populations of the own column (both sites): up(z-1), up(z), dn(z), rest(z), new plane's
  float2 up_m1 = f2c(0.f), up_0 = f2c(0.f), dn_0 = f2c(0.f), rest_0 = f2c(0.f);
  float2 up_new = f2c(0.f), dn_new = f2c(0.f), rest_new = f2c(0.f);
  // solid flags of both sites (bit 0: row 2 kp, bit 1: row 2 kp + 1) at z-1, z and the new plane
  unsigned sol_m1 = 0u, sol_0 = 0u, sol_new = 0u, sol_pref = 0u;
  int g2m = 0, g20 = G2, g2p = 2 * G2;

  auto load_mask = [&](int zp) -> unsigned {
    if constexpr (MASK) {
      const uint8_t* mz = a.mask + (long long)wrap(zp, a.nz) * plane;
      return (__ldg(mz + col0) != 0 ? 1u : 0u) | (__ldg(mz + col1) != 0 ? 2u : 0u);
    } else {
      (void)zp;
      return 0u;
    }
  };

  // staging: post-collision populations of plane p (both sites) into the ring
  auto stage = [&](auto par_c, int p, int g2, unsigned solid) -> bool {
    constexpr int par = decltype(par_c)::value;
    float2 m[10];
    read_raw(p, kRawStages == 2 ? par : (p - pbase) % kRawStages, m);
    const PostColl2 P = post_collision2(m, hx2, hy2, hz2, omm2);
    float* w0 = ring + R::base(0) + (R::NS0 == 2 ? par : 0) * G0 + ob;
    float* w1 = ring + R::base(1) + par * G1 + ob;
    float* w2 = ring + R::base(2) + g2 + ob;
    auto put = [&](auto qc, float2 v) {
      constexpr int q = decltype(qc)::value;
      if constexpr (q == QUP) {
        up_new = v;
      } else if constexpr (q == QDN) {
        dn_new = v;
      } else {
        constexpr int g = D::group(q);
        float* b = (g == 0 ? w0 : (g == 1 ? w1 : w2)) + D::gidx(q) * SITES;
        LBF_CHECK(a.flags, b - ring >= 0 && b - ring + 1 < R::VALUES);
        *reinterpret_cast<float2*>(b) = v;
      }
    };
    static_for<Q>([&](auto qc) {
      constexpr int q = decltype(qc)::value;
      if constexpr (q == QREST) {
        rest_new = P.q0;
      } else if constexpr (q < L::opp(q)) {
        float2 fq, fo;
        pop_pair2<L, q>(P, fq, fo);
        put(qc, fq);
        put(std::integral_constant<int, L::opp(q)>{}, fo);
      }
    });
    if constexpr (MASK) {
      LBF_CHECK(a.flags, g2 / GS2 + ob >= 0 && g2 / GS2 + ob + 1 < 3 * SITES);
      *reinterpret_cast<uint16_t*>(msk + g2 / GS2 + ob) = uint16_t((solid & 1u) | ((solid & 2u) << 7));
    }
    sol_new = solid;
    return solid != 0u;
  };

  float2 red[6] = {f2c(0.f), f2c(0.f), f2c(0.f), f2c(0.f), f2c(0.f), f2c(0.f)};

  if (me == 0) {
    abort_flag = 0;
    for (int s = 0; s < kRawStages; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
  }
  // ring slack read by the halo sites of the first and last pair: keep it finite (their results
  // are discarded, but the conservation sums mask them by multiplication)
  for (int i = me; i < kP2Pad; i += NT) {
    if constexpr (!MASK) ring[-kP2Pad + i] = 0.0f;
    ring[R::VALUES + i] = 0.0f;
  }
  __syncthreads();
  if (me == 0) {
    prefetch_tensormap(&tmap);
    for (int p = pbase; p < pbase + kRawStages; ++p) issue(p);
  }

  // prologue: stage planes z0-1 and z0
  sol_pref = load_mask(z0 - 1);
  wait_plane(z0 - 1);
  bool any_m = stage(std::integral_constant<int, 0>{}, z0 - 1, g2m, sol_pref);
  up_m1 = up_new;
  sol_m1 = sol_new;
  sol_pref = load_mask(z0);
  if constexpr (MASK)
    any_m = __syncthreads_or(any_m);
  else
    __syncthreads();
  if (me == 0) issue(z0 - 1 + kRawStages);
  wait_plane(z0);
  bool any_0 = stage(std::integral_constant<int, 1>{}, z0, g20, sol_pref);
  up_0 = up_new;
  dn_0 = dn_new;
  rest_0 = rest_new;
  sol_0 = sol_new;
  sol_pref = load_mask(z0 + 1);
  if (me == 0) wait_plane(z0 + 1);  // staged by the first iteration (z0 + 1 <= z1)
  if constexpr (MASK)
    any_0 = __syncthreads_or(any_0);
  else
    __syncthreads();
  if (me == 0) issue(z0 + kRawStages);

  // one plane: stage z+1, outputs of z. PAR = (z - z0) & 1 at compile time
  auto iteration = [&](auto par_c, int z) {
    constexpr int PAR = decltype(par_c)::value;
    // plane z+1 has landed: thread 0 waited for it before the barrier that ended the previous
    // iteration (or the prologue), and that barrier orders the observation for everyone
    bool any_p = stage(std::integral_constant<int, PAR>{}, z + 1, g2p, sol_pref);
    sol_pref = load_mask(z + 2);  // in flight during the outputs of plane z
    if constexpr (MASK)
      any_p = __syncthreads_or(any_p);
    else
      __syncthreads();
    if (me == 0) issue(z + 1 + kRawStages);  // the stage of plane z+1 was consumed by everyone

    // pull bases: group c_z = -1 from plane z+1, c_z = 0 from plane z, c_z = +1 from plane z-1
    const float* P0 = ring + R::base(0) + (R::NS0 == 2 ? PAR : 0) * G0 + ob;
    const float* P1 = ring + R::base(1) + (PAR ^ 1) * G1 + ob;
    const float* P2 = ring + R::base(2) + g2m + ob;
    auto gather = [&](auto walls_c) {
      constexpr bool W = decltype(walls_c)::value;
      const float* O0 = ring + R::base(0) + (R::NS0 == 2 ? (PAR ^ 1) : 0) * G0 + ob;  // own plane z (walls)
      const float* O2 = ring + R::base(2) + g20 + ob;
      const uint8_t* MM = msk + g2m / GS2 + ob;
      const uint8_t* M0 = msk + g20 / GS2 + ob;
      const uint8_t* MP = msk + g2p / GS2 + ob;
      const float wr = float(L::w(QREST));
      Accum2S A = {mul2(f2c(wr), rest_0), f2c(0.f), f2c(0.f), f2c(0.f), f2c(0.f),
                   f2c(0.f),              f2c(0.f), f2c(0.f), f2c(0.f), f2c(0.f)};
      // f_q at both sites: from (x - c_x, y - c_y) of its plane; rows 2 kp - c_y and 2 kp + 1 - c_y
      auto pulled = [&](auto qc) -> float2 {
        constexpr int q = decltype(qc)::value;
        constexpr int cx = L::cx(q), cy = L::cy(q), cz = L::cz(q);
        constexpr int g = D::group(q);
        const float* b = (g == 0 ? P0 : (g == 1 ? P1 : P2)) + D::gidx(q) * SITES - 2 * cx;
        constexpr int o0 = cy == 0 ? 0 : (cy > 0 ? -63 : 1);   // row 2 kp - c_y
        constexpr int o1 = cy == 0 ? 1 : (cy > 0 ? 0 : 64);    // row 2 kp + 1 - c_y
        LBF_CHECK(a.flags, (b + o0) - ring >= -FRONT && (b + o1) - ring < R::VALUES + kP2Pad);
        float2 v;
        if constexpr (cy == 0) {
          v = *reinterpret_cast<const float2*>(b);
        } else {
          v.x = b[o0];
          v.y = b[o1];
        }
        if constexpr (W) {
          const uint8_t* mk = (cz > 0 ? MM : (cz < 0 ? MP : M0)) - 2 * cx;
          LBF_CHECK(a.flags, (mk + o0) - msk >= -kP2Pad && (mk + o1) - msk < 3 * SITES + kP2Pad * 4);
          const bool s0 = mk[o0] != 0, s1 = mk[o1] != 0;
          if (s0 || s1) {  // halfway bounce-back: own post-collision population of opp(q)
            constexpr int o = L::opp(q);
            constexpr int go = D::group(o);
            const float2 own = *reinterpret_cast<const float2*>((go == 0 ? O0 : (go == 1 ? P1 : O2)) + D::gidx(o) * SITES);
            if (s0) v.x = own.x;
            if (s1) v.y = own.y;
          }
        }
        return v;
      };
      static_for<Q>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        if constexpr (q != QREST && q < L::opp(q) && q != QUP && q != QDN) {
          const float2 fq = pulled(qc);
          const float2 fo = pulled(std::integral_constant<int, L::opp(q)>{});
          accumulate_pair2<L::cx(q), L::cy(q), L::cz(q)>(A, fq, fo, float(L::w(q)));
        }
      });
      // axial pair: (0,0,+1) comes from the plane below, (0,0,-1) from the plane above
      float2 fup = up_m1, fdn = dn_new;
      if constexpr (W) {
        if (sol_m1 & 1u) fup.x = dn_0.x;
        if (sol_m1 & 2u) fup.y = dn_0.y;
        if (sol_new & 1u) fdn.x = up_0.x;
        if (sol_new & 2u) fdn.y = up_0.y;
      }
      accumulate_pair2<0, 0, 1>(A, fup, fdn, float(L::w(QUP)));
      return A;
    };
    Accum2S A;
    if constexpr (MASK) {
      if (any_m || any_0 || any_p)
        A = gather(std::true_type{});
      else
        A = gather(std::false_type{});
    } else {
      A = gather(std::false_type{});
    }
    // Eq. (corr): u = a1 + F/(2 rho), a2 = (sum c c f - cs2 a0 delta) + (u F + F u)/(2 rho)
    const float2 ux = add2(A.jx, hx2), uy = add2(A.jy, hy2), uz = add2(A.jz, hz2);
    const float2 a0c = mul2(f2c(1.0f / 3.0f), A.a0);
    // N_aa = (r_aa - a0/3) + u_a (2 h_a - u_a),  N_ab = r_ab + u_a (h_b - u_b) + h_a u_b
    const float2 nxx = fma2(ux, sub2(tx2, ux), sub2(A.rxx, a0c));
    const float2 nyy = fma2(uy, sub2(ty2, uy), sub2(A.ryy, a0c));
    const float2 nzz = fma2(uz, sub2(tz2, uz), sub2(A.rzz, a0c));
    const float2 nxy = fma2(ux, sub2(hy2, uy), fma2(hx2, uy, A.rxy));
    const float2 nxz = fma2(ux, sub2(hz2, uz), fma2(hx2, uz, A.rxz));
    const float2 nyz = fma2(uy, sub2(hz2, uz), fma2(hy2, uz, A.ryz));
    const float2 uu = fma2(ux, ux, fma2(uy, uy, mul2(uz, uz)));
    const bool w0 = out0 && !(sol_0 & 1u), w1 = out1 && !(sol_0 & 2u);
    const long long zp = (long long)z * plane;
    if (w0) {
      const long long zc = zp + col0;
      LBF_CHECK(a.flags, z >= 0 && z < a.nz && zc + 9 * N < 10 * N);
      dst[zc] = A.a0.x;
      dst[zc + N] = ux.x;
      dst[zc + 2 * N] = uy.x;
      dst[zc + 3 * N] = uz.x;
      dst[zc + 4 * N] = nxx.x;
      dst[zc + 5 * N] = nyy.x;
      dst[zc + 6 * N] = nzz.x;
      dst[zc + 7 * N] = nxy.x;
      dst[zc + 8 * N] = nxz.x;
      dst[zc + 9 * N] = nyz.x;
      if (!(uu.x <= a.umax2)) atomicOr(a.flags, 1u);
    }
    if (w1) {
      const long long zc = zp + col1;
      LBF_CHECK(a.flags, z >= 0 && z < a.nz && zc + 9 * N < 10 * N);
      dst[zc] = A.a0.y;
      dst[zc + N] = ux.y;
      dst[zc + 2 * N] = uy.y;
      dst[zc + 3 * N] = uz.y;
      dst[zc + 4 * N] = nxx.y;
      dst[zc + 5 * N] = nyy.y;
      dst[zc + 6 * N] = nzz.y;
      dst[zc + 7 * N] = nxy.y;
      dst[zc + 8 * N] = nxz.y;
      dst[zc + 9 * N] = nyz.y;
      if (!(uu.y <= a.umax2)) atomicOr(a.flags, 1u);
    }
    // conservation sums over the written sites (the discarded sites are finite: masked by 0)
    const float2 wm = make_float2(w0 ? 1.0f : 0.0f, w1 ? 1.0f : 0.0f);
    red[0] = fma2(wm, A.a0, red[0]);
    red[1] = fma2(wm, ux, red[1]);
    red[2] = fma2(wm, uy, red[2]);
    red[3] = fma2(wm, uz, red[3]);
    red[5] = fma2(wm, uu, red[5]);

    // rotate the own-column carries and the three-slot offsets to plane z+1
    up_m1 = up_0;
    up_0 = up_new;
    dn_0 = dn_new;
    rest_0 = rest_new;
    sol_m1 = sol_0;
    sol_0 = sol_new;
    any_m = any_0;
    any_0 = any_p;
    const int g2t = g2m;
    g2m = g20;
    g20 = g2p;
    g2p = g2t;
    if (me == 0 && z + 2 <= z1) wait_plane(z + 2);  // staged by the next iteration
    __syncthreads();
  };

  for (int z = z0; z < z1 && !abort_flag; z += 2) {
    iteration(std::integral_constant<int, 0>{}, z);
    if (z + 1 < z1 && !abort_flag) iteration(std::integral_constant<int, 1>{}, z + 1);
  }

  // after an aborted wait, let the copies still in flight land before the CTA exits (bounded)
  if (abort_flag && me == 0) {
    for (int p = max(pbase, issued - kRawStages + 1); p <= issued; ++p) {
      const int s = (p - pbase) % kRawStages;
      mbar_wait_bounded(&bars[s], uint32_t((p - pbase) / kRawStages) & 1u, kWaitPolls);
    }
  }

  if (a.partials != nullptr) {
    // warp sums in FP32, block and grid sums in FP64 (scratch: the idle ring)
    double* red_s = reinterpret_cast<double*>(smem_raw + RAW_BYTES);
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      float v = red[c].x + red[c].y;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red_s[kp * 6 + c] = static_cast<double>(v);
    }
    __syncthreads();
    const long long nb = (long long)gridDim.x * gridDim.y * gridDim.z;
    if (me < 6) {
      double s = 0.0;
      for (int r = 0; r < P2Tile<BY>::PAIRS; ++r) s += red_s[r * 6 + me];
      const long long b = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
      a.partials[b * 8 + me] = s;
    }
    // second stage in the same launch: the last block to finish sums the partials in a fixed order
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (me == 0) last = atomicAdd(a.counter, 1u) == (unsigned)(nb - 1);
    __syncthreads();
    if (last) {
      __threadfence();
      double* tree = reinterpret_cast<double*>(smem_raw);
      for (int i = me; i < 6 * 512; i += NT) tree[i] = 0.0;
      __syncthreads();
      for (int c = 0; c < 6; ++c) {
        double acc = 0.0;
        for (long long b = me; b < nb; b += NT) acc += __ldcg(a.partials + b * 8 + c);
        tree[c * 512 + me] = acc;
      }
      __syncthreads();
      for (int h = 256; h > 0; h >>= 1) {
        for (int i = me; i < 6 * h; i += NT) {
          const int c = i / h, j = i % h;
          tree[c * 512 + j] += tree[c * 512 + j + h];
        }
        __syncthreads();
      }
      if (me < 6) a.sums[me] = tree[me * 512];
      if (me == 0) *a.counter = 0u;
    }
  }
}

}  // namespace lbf
