// Fused pull-stream-and-collide step on line-aligned tiles with TMA tensor stores.
//
// Same method and arithmetic as k_stream_collide (Sec. 2, Eq. (pullLLB) followed by Eq. (corr);
// the helpers post_collision / pop_pair / full_populations / accumulate_* are shared), with a
// tile layout chosen for the GB300 memory system:
//   * a CTA owns 32 x TY output sites per plane: x0 = 32 bx is a multiple of 32, so one output row
//     of one field is one 128-byte line in FP32 (64 bytes in 16-bit storage) and the whole output
//     plane patch [10][TY][32] leaves shared memory as ONE TMA tensor store (cp.async.bulk.tensor,
//     bulk group) instead of ten per-thread stores per site, which no longer take issue slots or
//     straddle two lines;
//   * warps 0 .. TY-1 stage and output one row each (lane = x); warps TY and TY+1 stage the y halo
//     rows below and above the tile, only along the directions pulled into it (c_y = +1 / -1);
//     warp TY+2 stages the x halo columns (lanes 0 .. TY+1: x0 - 1, directions with c_x = +1;
//     lanes 16 .. 17+TY: x0 + 32, c_x = -1) and lane 31 of it issues every TMA copy and waits for
//     the next plane's load, so no output warp carries control work;
//   * the population ring holds rows of 34 sites (x0 - 1 .. x0 + 32), the TMA load box of a plane
//     is all 10 fields x (TY + 2) rows x (32 + 2 A) columns from x0 - A (A = 16 bytes / element).
// Planes whose patch holds a solid site (block-uniform) write their outputs with per-thread
// stores that skip solid sites (solid sites keep their moments); all other planes use the TMA
// store. Everything else (ring split by c_z, axial directions in registers, pairwise or packed
// accumulation, fused FP64 sums, bounded mbarrier waits) is as in k_stream_collide.
#pragma once

#include "stream_collide.cuh"

namespace lbf {

template <class S, int TY>
struct AlTile {
  static constexpr int XOUT = 32;                // outputs per row
  static constexpr int RW = XOUT + 2;            // ring row: x halo on both sides
  static constexpr int ROWS = TY + 2;            // ring rows: y halo on both sides
  static constexpr int SITES = RW * ROWS;        // ring sites of one plane
  static constexpr int A = 16 / int(sizeof(S));  // TMA x alignment in elements
  static constexpr int BX = XOUT + 2 * A;        // load box width, from x0 - A
  static constexpr int WARPS = TY + 3;
  static constexpr int THREADS = 32 * WARPS;
  static constexpr int CTRL = TY + 2;            // the x-halo / control warp
  static_assert(TY + 2 <= 16, "the x-halo warp stages both columns in two half-warps");
};

// population ring split by c_z over SITES sites per plane (as GroupRing)
template <class L, int SITES_, bool MASK>
struct RingN {
  using D = Dirs<L>;
  static constexpr int SITES = SITES_;
  static constexpr int NS0 = MASK ? 2 : 1, NS1 = 2, NS2 = 3;
  __host__ __device__ static constexpr int base(int g) {
    return g == 0 ? 0 : (g == 1 ? NS0 * D::gsize(0) * SITES : (NS0 * D::gsize(0) + NS1 * D::gsize(1)) * SITES);
  }
  static constexpr int VALUES = (NS0 * D::gsize(0) + NS1 * D::gsize(1) + NS2 * D::gsize(2)) * SITES;
};

constexpr size_t round128(size_t b) { return (b + 127) / 128 * 128; }

// output planes leave shared memory by TMA tensor stores (1) or by per-thread stores (0); with
// TMA stores, LBF_AL_OUT_STAGES output stages rotate so that a store may still be reading one
// stage while the next plane is written into the other
#ifndef LBF_AL_TMA_STORE
#define LBF_AL_TMA_STORE 0
#endif
#ifndef LBF_AL_OUT_STAGES
#define LBF_AL_OUT_STAGES 1
#endif
// halo rows and columns stage only the directions pulled into the tile (0) or every direction
// with the output rows' code (1)
// with walls, one gather body whose bounce-back selects run on every tile (1), or a second body
// without them for tiles far from any wall (0)
#ifndef LBF_AL_ONE_GATHER
#define LBF_AL_ONE_GATHER 0
#endif
#ifndef LBF_AL_HALO_ALL
#define LBF_AL_HALO_ALL 1
#endif
constexpr int kAlOutStages = LBF_AL_TMA_STORE ? LBF_AL_OUT_STAGES : 0;

template <class S, int TY>
constexpr size_t al_stage_bytes() {
  return round128(size_t(10) * AlTile<S, TY>::ROWS * AlTile<S, TY>::BX * sizeof(S));
}
template <class S, int TY>
constexpr size_t al_out_bytes() {
  return kAlOutStages * round128(size_t(10) * TY * 32 * sizeof(S));
}

template <class L, class S, int TY, bool MASK>
constexpr size_t al_smem_bytes() {
  using T = typename ComputeOf<S>::type;
  using G = AlTile<S, TY>;
  return 128 + size_t(kRawStages) * al_stage_bytes<S, TY>() + al_out_bytes<S, TY>() +
         size_t(RingN<L, G::SITES, MASK>::VALUES + 2 * kRingPad) * sizeof(T) +
         (MASK ? size_t(3) * G::SITES + 2 * kRingPad : 0);
}

// output rows per CTA and minimum resident CTAs of the aligned kernel, per lattice, storage width,
// walls and basis (tuning defines LBF_AL_ROWS_*). D3Q19 FP32: 8 rows without walls (the tallest
// tile at 3 CTAs/SM, 75.9 KB; 64.9 GLUPS at 512^3 against 58.4 for 6 rows and 60.5 / 60.9 for 5 / 7),
// 7 rows with walls (the solid-flag ring and the second c_z = -1 slot need 3 KB more per CTA)
#ifndef LBF_AL_ROWS_Q19
#define LBF_AL_ROWS_Q19 7
#endif
#ifndef LBF_AL_ROWS_Q19_NM
#define LBF_AL_ROWS_Q19_NM 8
#endif
#ifndef LBF_AL_ROWS_Q19_16
#define LBF_AL_ROWS_Q19_16 8
#endif
#ifndef LBF_AL_ROWS_Q27
#define LBF_AL_ROWS_Q27 6
#endif
#ifndef LBF_AL_ROWS_Q27_NM
#define LBF_AL_ROWS_Q27_NM 8
#endif
#ifndef LBF_AL_ROWS_Q27_16
#define LBF_AL_ROWS_Q27_16 6
#endif
#ifndef LBF_AL_ROWS_Q27H_16
#define LBF_AL_ROWS_Q27H_16 5
#endif
constexpr int al_rows(int Q, int bytes, bool mask, bool high) {
  return Q == 19 ? (bytes == 4 ? (mask ? LBF_AL_ROWS_Q19 : LBF_AL_ROWS_Q19_NM) : LBF_AL_ROWS_Q19_16)
                 : (bytes == 4 ? (mask ? LBF_AL_ROWS_Q27 : LBF_AL_ROWS_Q27_NM)
                               : (high ? LBF_AL_ROWS_Q27H_16 : LBF_AL_ROWS_Q27_16));
}
// CTAs per SM that fit the shared memory (228 KB per SM, 1 KB reserved per CTA), at most 4
template <class L, class S, int TY, bool MASK>
constexpr int al_minb() {
  constexpr size_t per = al_smem_bytes<L, S, TY, MASK>() + 1024 + 64;
  constexpr int n = int((size_t(228) * 1024) / per);
  return n < 1 ? 1 : (n > 4 ? 4 : n);
}

template <class L, class S, int TY, bool MASK, bool FF, bool RN>
__global__ void __launch_bounds__(AlTile<S, TY>::THREADS, al_minb<L, S, TY, MASK>())
    k_stream_collide_al(const FwdParams a, const __grid_constant__ CUtensorMap tload,
                        const __grid_constant__ CUtensorMap tstore) {
  using T = typename ComputeOf<S>::type;
  using G = AlTile<S, TY>;
  using D = Dirs<L>;
  using R = RingN<L, G::SITES, MASK>;
  constexpr int Q = L::Q;
  constexpr int RW = G::RW, SITES = G::SITES, BX = G::BX, AL = G::A, ROWS = G::ROWS;
  constexpr int QREST = D::find(0, 0, 0);
  constexpr int QUP = D::find(0, 0, 1);
  constexpr int QDN = D::find(0, 0, -1);
  constexpr int STAGE_ELEMS = 10 * ROWS * BX;
  constexpr int STAGE_STRIDE = int(al_stage_bytes<S, TY>() / sizeof(S));
  constexpr size_t RAW_BYTES = size_t(kRawStages) * al_stage_bytes<S, TY>();
  constexpr size_t OUT_BYTES = al_out_bytes<S, TY>();
  constexpr int G0 = D::gsize(0) * SITES, G1 = D::gsize(1) * SITES, G2 = D::gsize(2) * SITES;
  constexpr int GS2 = D::gsize(2);
  constexpr int OSTR = TY * 32;  // field stride of the output stage
  constexpr int OSTAGE = int(round128(size_t(10) * TY * 32 * sizeof(S)) / sizeof(S));  // elements per output stage
  static_assert(al_smem_bytes<L, S, TY, MASK>() >= 6 * 512 * sizeof(double) + 128, "smem too small for the final tree");
  static_assert(G::THREADS <= 512, "final tree assumes <= 512 threads");

  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* sbase = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  S* rawst = reinterpret_cast<S*>(sbase);
  S* outst = reinterpret_cast<S*>(sbase + RAW_BYTES);
  T* ring = reinterpret_cast<T*>(sbase + RAW_BYTES + OUT_BYTES) + kRingPad;
  uint8_t* msk = reinterpret_cast<uint8_t*>(ring + R::VALUES + kRingPad) + kRingPad;
  __shared__ __align__(8) uint64_t bars[kRawStages];
  __shared__ int abort_flag;

  const S* __restrict__ src = static_cast<const S*>(a.src);
  S* __restrict__ dst = static_cast<S*>(a.dst);
  const T* __restrict__ ffield = static_cast<const T*>(a.force_field);

  const int lane = threadIdx.x, warp = threadIdx.y;
  const int yb = a.y_begin, yrows = a.y_rows > 0 ? a.y_rows : a.ny;  // this launch's output rows
  const int x0 = blockIdx.x * 32, y0 = yb + int(blockIdx.y) * TY;     // y0 may exceed ny: wraps
  // this thread's staged site: ring row rr, ring column rc; role 0 = output row (every direction),
  // 1 / 2 = y halo below / above (c_y = +1 / -1), 3 / 4 = x halo left / right (c_x = +1 / -1),
  // 5 = nothing to stage
  int role, rr, rc;
  if (warp < TY) {
    role = 0, rr = warp + 1, rc = lane + 1;
  } else if (warp == TY) {
    role = 1, rr = 0, rc = lane + 1;
  } else if (warp == TY + 1) {
    role = 2, rr = ROWS - 1, rc = lane + 1;
  } else if (lane < 16) {
    role = lane < ROWS ? 3 : 5, rr = lane < ROWS ? lane : 0, rc = 0;
  } else {
    role = lane - 16 < ROWS ? 4 : 5, rr = lane - 16 < ROWS ? lane - 16 : 0, rc = RW - 1;
  }
  const bool ctrl = warp == G::CTRL && lane == 31;
  const int gx = x0 - 1 + rc;
  const int gy = y0 - 1 + rr;
  const int sx = ((gx % a.nx) + a.nx) % a.nx;
  const int sy = ((gy % a.ny) + a.ny) % a.ny;
  const bool out_row = warp < TY;  // warp-uniform
  const bool outcol = out_row && x0 + lane < a.nx && (y0 - yb) + warp < yrows;
  const bool inbox = gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny;  // TMA delivers this site
  const bool needed = role != 5 && gx <= a.nx && gy - yb <= yrows;    // read by some output
  const long long plane = (long long)a.nx * a.ny;
  const int col = sy * a.nx + sx;
  const long long N = a.N;
  const int z0 = blockIdx.z * a.zchunk;
  const int z1 = min(a.nz, z0 + a.zchunk);
  const int me = rr * RW + rc;  // ring site of this thread
  const T one_m_omega = T(1) - pick<T>(a.omega, a.omega_f);
  const T Fu0 = pick<T>(a.force[0], a.force_f[0]), Fu1 = pick<T>(a.force[1], a.force_f[1]),
          Fu2 = pick<T>(a.force[2], a.force_f[2]);
  const int pbase = z0 - 1;
  const S* raw_me = rawst + rr * BX + (rc - 1 + AL);

  int issued = pbase - 1;
  auto issue = [&](int p) {  // control thread only
    if (p > z1 || abort_flag) return;
    const int s = (p - pbase) % kRawStages;
    S* dstp = rawst + s * STAGE_STRIDE;
    if ((smem_u32(dstp) & 127u) != 0u) {
      atomicOr(a.flags, 4u);
      abort_flag = 1;
      return;
    }
    LBF_CHECK(a.flags, ((x0 - AL) * int(sizeof(S))) % 16 == 0 && s >= 0 && s < kRawStages);
    mbar_arrive_expect_tx(&bars[s], uint32_t(STAGE_ELEMS * sizeof(S)));
    tma_load_4d(dstp, &tload, &bars[s], x0 - AL, y0 - 1, wrap(p, a.nz), 0);
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

  auto load_extra = [&](int zp, SiteExtra<T, false>& e) {
    const long long zoff = (long long)wrap(zp, a.nz) * plane;
    if constexpr (FF) {
      if (needed) {
        const T* fb = ffield + zoff;
        e.F[0] = Fu0 + __ldg(fb + col);
        e.F[1] = Fu1 + __ldg(fb + N + col);
        e.F[2] = Fu2 + __ldg(fb + 2 * N + col);
      } else {
        e.F[0] = Fu0, e.F[1] = Fu1, e.F[2] = Fu2;
      }
    }
    if constexpr (MASK) e.solid = needed && __ldg(a.mask + zoff + col) != 0;
    else e.solid = false;
  };

  auto read_raw = [&](int p, int st, T (&m)[10]) {
    if (inbox) {
      const S* b = raw_me + st * STAGE_STRIDE;
      LBF_CHECK(a.flags, st >= 0 && st < kRawStages && rc - 1 + AL >= 0 && rc - 1 + AL < BX &&
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
    } else if (needed) {
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

  T Fown[3] = {Fu0, Fu1, Fu2}, Fnext[3] = {Fu0, Fu1, Fu2};
  T up_m1 = T(0), up_0 = T(0), dn_0 = T(0), rest_0 = T(0);
  T up_new = T(0), dn_new = T(0), rest_new = T(0);
  bool sol_m1 = false, sol_0 = false, sol_new = false;
  int g2m = 0, g20 = G2, g2p = 2 * G2;

  // staging of plane p by role H (compile time): the post-collision populations this site
  // contributes to the tile, into the ring (axial ones of output rows into registers)
  // par = (p - pbase) & 1 at run time: one copy of the plane loop (instruction-cache footprint)
  auto stage_as = [&](int par, auto role_c, int p, int g2, const SiteExtra<T, false>& e) {
    constexpr int H = decltype(role_c)::value;
    T m[10];
    read_raw(p, kRawStages == 2 ? par : (p - pbase) % kRawStages, m);
    T omm = one_m_omega;
    if constexpr (FF) {
      if (H == 0) {
        Fnext[0] = e.F[0];
        Fnext[1] = e.F[1];
        Fnext[2] = e.F[2];
      }
    }
    const T Fs0 = FF ? e.F[0] : Fu0, Fs1 = FF ? e.F[1] : Fu1, Fs2 = FF ? e.F[2] : Fu2;
    if constexpr (Codec<S>::scaled) omm *= a.sc.dec[2];
    T* w0 = ring + R::base(0) + (R::NS0 == 2 ? par : 0) * G0 + me;
    T* w1 = ring + R::base(1) + par * G1 + me;
    T* w2 = ring + R::base(2) + g2 + me;
    auto wanted = [](int q) {
      return H == 0 || (H == 1 && L::cy(q) == 1) || (H == 2 && L::cy(q) == -1) || (H == 3 && L::cx(q) == 1) ||
             (H == 4 && L::cx(q) == -1);
    };
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
      const T hv[3] = {Fs0 * T(0.5), Fs1 * T(0.5), Fs2 * T(0.5)};
      const T Nt[3][3] = {{m[4], m[7], m[8]}, {m[7], m[5], m[9]}, {m[8], m[9], m[6]}};
      T g[27];
      full_populations<T>(m[0], uv, hv, Nt, omm, g);
      static_for<Q>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        if constexpr (q == QREST) {
          if constexpr (H == 0) rest_new = g[q];
        } else if constexpr (wanted(q)) {
          put(qc, g[q]);
        }
      });
    } else {
      const PostColl<T> P = post_collision<T>(m[0], m[1], m[2], m[3], m[4], m[5], m[6], m[7], m[8], m[9], Fs0, Fs1,
                                              Fs2, T(0.5), omm);
      static_for<Q>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        constexpr bool need_q = wanted(q), need_o = wanted(L::opp(q));
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
    if (H == 0) sol_new = e.solid;
  };
  auto stage = [&](int par_c, int p, int g2, const SiteExtra<T, false>& e) -> bool {
#if LBF_AL_HALO_ALL
    // one staging body for every role (every direction): less code than the per-role bodies
    if (role != 5) stage_as(par_c, std::integral_constant<int, 0>{}, p, g2, e);
    return e.solid;
#endif
    if (warp < TY) stage_as(par_c, std::integral_constant<int, 0>{}, p, g2, e);
    else if (warp == TY) stage_as(par_c, std::integral_constant<int, 1>{}, p, g2, e);
    else if (warp == TY + 1) stage_as(par_c, std::integral_constant<int, 2>{}, p, g2, e);
    else if (role == 3) stage_as(par_c, std::integral_constant<int, 3>{}, p, g2, e);
    else if (role == 4) stage_as(par_c, std::integral_constant<int, 4>{}, p, g2, e);
    return e.solid;
  };

  T red[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
  SiteExtra<T, false> ex;
  ex.solid = false;

  if (ctrl) {
    abort_flag = 0;
    for (int s = 0; s < kRawStages; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
  }
  if constexpr (MASK) {
    for (int i = warp * 32 + lane; i < kRingPad; i += G::THREADS) {
      msk[-kRingPad + i] = 0;
      msk[3 * SITES + i] = 0;
    }
  }
  __syncthreads();
  if (ctrl) {
    prefetch_tensormap(&tload);
    prefetch_tensormap(&tstore);
    for (int p = pbase; p < pbase + kRawStages; ++p) issue(p);
  }

  load_extra(z0 - 1, ex);
  wait_plane(z0 - 1);
  bool any_m = stage(0, z0 - 1, g2m, ex);
  up_m1 = up_new;
  sol_m1 = sol_new;
  load_extra(z0, ex);
  if constexpr (MASK)
    any_m = __syncthreads_or(any_m);
  else
    __syncthreads();
  if (ctrl) issue(z0 - 1 + kRawStages);
  wait_plane(z0);
  bool any_0 = stage(1, z0, g20, ex);
  if (warp == G::CTRL) wait_plane(z0 + 1);
  up_0 = up_new;
  dn_0 = dn_new;
  rest_0 = rest_new;
  sol_0 = sol_new;
  Fown[0] = Fnext[0];
  Fown[1] = Fnext[1];
  Fown[2] = Fnext[2];
  load_extra(z0 + 1, ex);
  if constexpr (MASK)
    any_0 = __syncthreads_or(any_0);
  else
    __syncthreads();
  if (ctrl) issue(z0 + kRawStages);

  bool store_pending = false;  // control thread: a TMA store may still read the output stage

  auto iteration = [&](int PAR, int z) {
    bool any_p = stage(PAR, z + 1, g2p, ex);
    load_extra(z + 2, ex);
    if (ctrl && store_pending) {
      // the output stage written after the barrier is free: with one stage the store issued last,
      // with two the one before it has finished reading shared memory
      if constexpr (kAlOutStages >= 2)
        bulk_wait_group_read1();
      else
        bulk_wait_group_read0();
    }
    if constexpr (MASK)
      any_p = __syncthreads_or(any_p);
    else
      __syncthreads();
    if (ctrl) issue(z + 1 + kRawStages);
    // block-uniform: a solid site in this plane's patch (then per-thread stores that skip solid
    // sites); without TMA stores every plane takes that path
    const bool wall = !LBF_AL_TMA_STORE || (MASK && (any_0 != 0));
    S* const ostage = outst + (kAlOutStages >= 2 ? ((z - z0) & 1) * OSTAGE : 0);
    if (out_row) {
      const T* P0 = ring + R::base(0) + (R::NS0 == 2 ? PAR : 0) * G0 + me;
      const T* P1 = ring + R::base(1) + (PAR ^ 1) * G1 + me;
      const T* P2 = ring + R::base(2) + g2m + me;
      auto gather = [&](auto walls_c) {
        constexpr bool W = decltype(walls_c)::value;
        const T* O0 = ring + R::base(0) + (R::NS0 == 2 ? (PAR ^ 1) : 0) * G0 + me;
        const T* O2 = ring + R::base(2) + g20 + me;
        const uint8_t* MM = msk + g2m / GS2 + me;
        const uint8_t* M0 = msk + g20 / GS2 + me;
        const uint8_t* MP = msk + g2p / GS2 + me;
        Accum<T> A = {T(L::w(QREST)) * rest_0, T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
        auto pulled = [&](auto qc) -> T {
          constexpr int q = decltype(qc)::value;
          constexpr int cx = L::cx(q), cy = L::cy(q), cz = L::cz(q);
          constexpr int g = D::group(q);
          constexpr int off = D::gidx(q) * SITES - cy * RW - cx;
          LBF_CHECK(a.flags, ((g == 0 ? P0 : (g == 1 ? P1 : P2)) + off) - ring >= 0 &&
                                 ((g == 0 ? P0 : (g == 1 ? P1 : P2)) + off) - ring < R::VALUES);
          T v = (g == 0 ? P0 : (g == 1 ? P1 : P2))[off];
          if constexpr (W) {
            const uint8_t* mk = cz > 0 ? MM : (cz < 0 ? MP : M0);
            LBF_CHECK(a.flags, (mk - cy * RW - cx) - msk >= 0 && (mk - cy * RW - cx) - msk < 3 * SITES);
            if (mk[-cy * RW - cx]) {
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
        T fup = up_m1, fdn = dn_new;
        if constexpr (W) {
          if (sol_m1) fup = dn_0;
          if (sol_new) fdn = up_0;
        }
        accumulate_pair<0, 0, 1, T>(A, fup, fdn, T(L::w(QUP)));
        return A;
      };
      Accum<T> A;
      if constexpr (MASK && LBF_AL_ONE_GATHER) {
        A = gather(std::true_type{});  // one gather body: the bounce-back selects run everywhere
      } else if constexpr (MASK) {
        if (any_m || any_0 || any_p)
          A = gather(std::true_type{});
        else
          A = gather(std::false_type{});
      } else {
        A = gather(std::false_type{});
      }
      // Eq. (corr): u = a1 + F/(2 rho), a2 = (sum c c f - cs2 a0 delta) + (u F + F u)/(2 rho), rho = 1
      const T hx = (FF ? Fown[0] : Fu0) * T(0.5), hy = (FF ? Fown[1] : Fu1) * T(0.5),
              hz = (FF ? Fown[2] : Fu2) * T(0.5);
      const T ux = A.jx + hx, uy = A.jy + hy, uz = A.jz + hz;
      const T a0c = A.a0 * (T(1) / T(3));
      const T nxx = (A.rxx - a0c) + T(2) * ux * hx - ux * ux;
      const T nyy = (A.ryy - a0c) + T(2) * uy * hy - uy * uy;
      const T nzz = (A.rzz - a0c) + T(2) * uz * hz - uz * uz;
      const T nxy = A.rxy + (ux * hy + hx * uy) - ux * uy;
      const T nxz = A.rxz + (ux * hz + hx * uz) - ux * uz;
      const T nyz = A.ryz + (uy * hz + hy * uz) - uy * uz;
      const T uu = ux * ux + uy * uy + uz * uz;
      const long long zc = (long long)z * plane + col;
      uint32_t rs = Codec<S>::scaled && !RN ? fmix32(uint32_t(zc) ^ a.salt) : 0u;
      if (!wall) {
        // every site of the patch is fluid: the output stage, stored by one TMA box after the barrier
        S* o = ostage + warp * 32 + lane;
        LBF_CHECK(a.flags, warp * 32 + lane + 9 * OSTR < 10 * OSTR);
        st_field<S, RN>(o, 0, A.a0, a.sc.enc[0], rs);
        st_field<S, RN>(o + OSTR, 0, ux, a.sc.enc[1], rs);
        st_field<S, RN>(o + 2 * OSTR, 0, uy, a.sc.enc[1], rs);
        st_field<S, RN>(o + 3 * OSTR, 0, uz, a.sc.enc[1], rs);
        st_field<S, true>(o + 4 * OSTR, 0, nxx, a.sc.enc[2], rs);
        st_field<S, true>(o + 5 * OSTR, 0, nyy, a.sc.enc[2], rs);
        st_field<S, true>(o + 6 * OSTR, 0, nzz, a.sc.enc[2], rs);
        st_field<S, true>(o + 7 * OSTR, 0, nxy, a.sc.enc[2], rs);
        st_field<S, true>(o + 8 * OSTR, 0, nxz, a.sc.enc[2], rs);
        st_field<S, true>(o + 9 * OSTR, 0, nyz, a.sc.enc[2], rs);
        fence_proxy_async_smem();
      } else if (outcol && !sol_0) {
        LBF_CHECK(a.flags, z >= 0 && z < a.nz && col >= 0 && col < plane && zc + 9 * N < 10 * N);
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
      if (outcol && !sol_0) {
        if (!(uu <= T(a.umax2))) atomicOr(a.flags, 1u);
        red[0] += A.a0;
        red[1] += ux;
        red[2] += uy;
        red[3] += uz;
        red[5] += uu;
      }
    }
    up_m1 = up_0;
    up_0 = up_new;
    dn_0 = dn_new;
    rest_0 = rest_new;
    sol_m1 = sol_0;
    sol_0 = sol_new;
    Fown[0] = Fnext[0];
    Fown[1] = Fnext[1];
    Fown[2] = Fnext[2];
    any_m = any_0;
    any_0 = any_p;
    const int g2t = g2m;
    g2m = g20;
    g20 = g2p;
    g2p = g2t;
    if (warp == G::CTRL && z + 2 <= z1) wait_plane(z + 2);
    __syncthreads();
    if (ctrl && !wall) {
      tma_store_4d(&tstore, ostage, x0, y0, z, 0);
      bulk_commit_group();
      store_pending = true;
    }
  };

  for (int z = z0; z < z1 && !abort_flag; ++z) iteration((z - z0) & 1, z);

  if (ctrl) {
    bulk_wait_group0();  // the stores are complete and the output stage is free
    if (abort_flag) {    // let the loads still in flight land before the CTA exits (bounded)
      for (int p = max(pbase, issued - kRawStages + 1); p <= issued; ++p) {
        const int s = (p - pbase) % kRawStages;
        mbar_wait_bounded(&bars[s], uint32_t((p - pbase) / kRawStages) & 1u, kWaitPolls);
      }
    }
  }
  __syncthreads();

  if (a.partials != nullptr) {
    double* red_s = reinterpret_cast<double*>(sbase + RAW_BYTES + OUT_BYTES);
    const int tid = warp * 32 + lane;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      T v = red[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red_s[warp * 6 + k] = static_cast<double>(v);
    }
    __syncthreads();
    const long long nb = (long long)gridDim.x * gridDim.y * gridDim.z;
    if (tid < 6) {
      double s = 0.0;
      for (int r = 0; r < G::WARPS; ++r) s += red_s[r * 6 + tid];
      const long long b = a.block_base + ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
      a.partials[b * 8 + tid] = s;
    }
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    const long long nall = a.final_blocks > 0 ? a.final_blocks : a.block_base + nb;  // partials to add
    if (tid == 0) last = atomicAdd(a.counter, 1u) == (unsigned)(a.final_blocks > 0 ? nall - 1 : nb - 1);
    __syncthreads();
    if (last) {
      __threadfence();
      constexpr int NT = G::THREADS;
      double* tree = reinterpret_cast<double*>(sbase);
      for (int i = tid; i < 6 * 512; i += NT) tree[i] = 0.0;
      __syncthreads();
      for (int k = 0; k < 6; ++k) {
        double acc = 0.0;
        for (long long b = tid; b < nall; b += NT) acc += __ldcg(a.partials + b * 8 + k);
        tree[k * 512 + tid] = acc;
      }
      __syncthreads();
      for (int h = 256; h > 0; h >>= 1) {
        for (int i = tid; i < 6 * h; i += NT) {
          const int k = i / h, j = i % h;
          tree[k * 512 + j] += tree[k * 512 + j + h];
        }
        __syncthreads();
      }
      if (tid < 6) a.sums[tid] = tree[tid * 512];
      if (tid == 0) *a.counter = 0u;
    }
  }
}

}  // namespace lbf
