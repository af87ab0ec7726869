// Fused pull-stream-and-collide step with row-level synchronisation.
//
// Same tile, ring and arithmetic as k_stream_collide (Sec. 2, Eq. (pullLLB) followed by
// Eq. (corr)): a CTA owns 30 x BY output sites per plane, warp r holds ring row r (rows 0 and
// BY+1 are the y halo), and the CTA marches along z. What changes is how the warps wait for each
// other. An output row only pulls populations from the ring rows r-1, r, r+1, so instead of two
// CTA-wide barriers per plane every row signals and waits on its neighbours through mbarriers:
//   staged[r]  completes a phase when row r has written its populations of the next plane;
//   done[r]    completes a phase when every output row that pulls from row r (r-1, r, r+1) has
//              finished a plane, which frees row r's ring slots of an older plane;
//   full[s]    completes when the TMA box of a plane (all rows) has landed in raw stage s; the
//              last row to finish reading a stage (a shared counter per stage) issues its refill
//              with the plane two ahead, so no row waits for the others to consume it.
// Row r stages plane p once done[r] reports output plane p - 2 (the ring keeps 2, 2 and 3 plane
// slots for the c_z = -1, 0, +1 groups: p - 2 is the newest plane whose slots plane p reuses), and
// outputs plane z once staged[r-1..r+1] report plane z + 1. Rows therefore drift by up to one
// plane, and a slow warp delays only its neighbours instead of the whole CTA. Phases never run
// two ahead of a waiter (each wait is for the current or the previous phase), so the parity of
// the plane index identifies them. Every wait is bounded: on time-out the row sets error bit 1
// (reported as LBF_EINTERNAL), raises the CTA's abort flag and leaves its loop; the other rows'
// waits see the flag and leave too.
// Walls: whether a CTA's patch (planes z0-1 .. z1) holds any solid site is decided on the host
// (tile_walls, one byte per CTA), which selects the bounce-back gather for the whole CTA.
#pragma once

#include "stream_collide.cuh"

namespace lbf {

// slack before and after the population and solid-flag rings: the edge lanes of the first and
// last output rows read one element beyond them (results discarded)
constexpr int kRowsPad = 8;

template <class L, class S, int BY, bool MASK>
constexpr size_t rows_smem_bytes() {
  using T = typename ComputeOf<S>::type;
  return 128 + size_t(kRawStages) * raw_stage_bytes<S, BY + 2>() +
         size_t(GroupRing<L, BY + 2, MASK>::VALUES + 2 * kRowsPad) * sizeof(T) +
         (MASK ? size_t(3) * (BY + 2) * 32 + 2 * kRowsPad : 0);
}

template <class L, class S, int BY, bool MASK, bool FF, bool RN>
__global__ void __launch_bounds__(FwdTile<BY>::THREADS, fwd_minb(L::Q, int(sizeof(S)), MASK, false))
    k_stream_collide_rows(const FwdParams a, const __grid_constant__ CUtensorMap tmap,
                          const uint8_t* __restrict__ tile_walls) {
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
  constexpr size_t RAW_BYTES = size_t(kRawStages) * raw_stage_bytes<S, ROWS>();
  constexpr int G0 = D::gsize(0) * SITES, G1 = D::gsize(1) * SITES, G2 = D::gsize(2) * SITES;
  constexpr int GS2 = D::gsize(2);
  static_assert(rows_smem_bytes<L, S, BY, MASK>() >= 6 * 512 * sizeof(double) + 128, "smem too small for the final tree");
  static_assert(FwdTile<BY>::THREADS <= 512, "final tree assumes <= 512 threads");

  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* sbase = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
  S* rawst = reinterpret_cast<S*>(sbase);
  T* ring = reinterpret_cast<T*>(sbase + RAW_BYTES) + kRowsPad;
  uint8_t* msk = reinterpret_cast<uint8_t*>(ring + R::VALUES + kRowsPad) + kRowsPad;
  __shared__ __align__(8) uint64_t full[kRawStages];
  __shared__ __align__(8) uint64_t staged[ROWS];
  __shared__ __align__(8) uint64_t done[ROWS];
  __shared__ int rawcnt[kRawStages];
  __shared__ volatile int abort_flag;

  const S* __restrict__ src = static_cast<const S*>(a.src);
  S* __restrict__ dst = static_cast<S*>(a.dst);
  const T* __restrict__ ffield = static_cast<const T*>(a.force_field);

  const int lane = threadIdx.x, row = threadIdx.y;
  const int x0 = blockIdx.x * FwdTile<BY>::XOUT;
  const int gx = x0 - 1 + lane;
  const int gy = blockIdx.y * BY - 1 + row;
  const int sx = ((gx % a.nx) + a.nx) % a.nx;
  const int sy = ((gy % a.ny) + a.ny) % a.ny;
  const bool out_row = row >= 1 && row <= BY;  // warp-uniform
  const bool outcol = out_row && lane >= 1 && lane <= FwdTile<BY>::XOUT && gx < a.nx && gy < a.ny;
  const bool inbox = gx >= 0 && gx < a.nx && gy >= 0 && gy < a.ny;
  const bool needed = gx <= a.nx && gy <= a.ny;
  const int xa = ((x0 - 1 + AL) / AL - 1) * AL;
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
  const int pbase = z0 - 1;
  const long long cta = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  const bool walls = MASK && (tile_walls == nullptr || tile_walls[cta] != 0);  // block-uniform

  // bounded wait on a phase parity, warp-uniform (every lane polls, the warp leaves together);
  // gives up on time-out, or when another row has aborted. The non-blocking test is used with a
  // short sleep between polls: a potentially blocking try_wait can suspend the warp for far
  // longer than a neighbour row needs to arrive, and a hot spin takes issue slots from the rows
  // doing the work.
  auto wait_bar = [&](uint64_t* bar, uint32_t parity) -> bool {
    for (uint32_t i = 0; i < kWaitPolls; ++i) {
      const bool ok = mbar_test_wait(bar, parity);
      if (__all_sync(0xffffffffu, ok)) return true;
      __nanosleep(32);
      if ((i & 63u) == 63u && __any_sync(0xffffffffu, abort_flag != 0)) return false;
    }
    if (lane == 0) {
      atomicOr(a.flags, 2u);
      abort_flag = 1;
    }
    return false;
  };
  auto arrive = [&](uint64_t* bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
  };

  int issued = pbase - 1;  // lane 0 of an issuing row: last plane it issued
  auto issue = [&](int p) {  // one lane of the CTA per plane
    if (p > z1 || abort_flag) return;
    const int s = (p - pbase) % kRawStages;
    S* dstp = rawst + s * STAGE_STRIDE;
    if ((smem_u32(dstp) & 127u) != 0u) {
      atomicOr(a.flags, 4u);
      abort_flag = 1;
      return;
    }
    LBF_CHECK(a.flags, (xa * int(sizeof(S))) % 16 == 0);
    mbar_arrive_expect_tx(&full[s], uint32_t(STAGE_ELEMS * sizeof(S)));
    tma_load_4d(dstp, &tmap, &full[s], xa, int(blockIdx.y) * BY - 1, wrap(p, a.nz), 0);
    issued = max(issued, p);
  };

  auto load_extra = [&](int zp, SiteExtra<T, 0>& e) {
    const long long zoff = (long long)wrap(zp, a.nz) * plane;
    if constexpr (FF) {
      const T* fb = ffield + zoff;
      e.F[0] = Fu0 + __ldg(fb + col);
      e.F[1] = Fu1 + __ldg(fb + N + col);
      e.F[2] = Fu2 + __ldg(fb + 2 * N + col);
    }
    if constexpr (MASK) e.solid = __ldg(a.mask + zoff + col) != 0;
    else e.solid = false;
  };

  auto read_raw = [&](int p, T (&m)[10]) {
    if (inbox) {
      const S* b = rawst + ((p - pbase) % kRawStages) * STAGE_STRIDE + row * BX + lane + xoff;
      LBF_CHECK(a.flags, lane + xoff < BX && (b - rawst) + 9 * ROWS * BX < kRawStages * STAGE_STRIDE);
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

  // staging of plane p by this row: wait for its box, read it, refill the stage with plane p + 2,
  // wait until the ring slots of plane p are free (output p - 2 done by the rows that read them),
  // write the populations, signal staged[row]
  auto stage = [&](auto par_c, int p, int g2, const SiteExtra<T, 0>& e) -> bool {
    constexpr int par = decltype(par_c)::value;
    const int s = (p - pbase) % kRawStages;
    if (!wait_bar(&full[s], uint32_t((p - pbase) / kRawStages) & 1u)) return false;
    T m[10];
    read_raw(p, m);
    __syncwarp();
    if (lane == 0) {
      // this row has read its part of the stage; the last row to do so refills it
      __threadfence_block();
      if (atomicAdd(&rawcnt[s], 1) == ROWS - 1) {
        rawcnt[s] = 0;
        __threadfence_block();
        issue(p + kRawStages);
      }
    }
    if (p - 2 >= z0 && !wait_bar(&done[row], uint32_t(p - 2 - z0) & 1u)) return false;
    T omm = one_m_omega;
    if constexpr (FF) {
      Fnext[0] = e.F[0];
      Fnext[1] = e.F[1];
      Fnext[2] = e.F[2];
    }
    const T Fs0 = FF ? e.F[0] : Fu0, Fs1 = FF ? e.F[1] : Fu1, Fs2 = FF ? e.F[2] : Fu2;
    if constexpr (Codec<S>::scaled) omm *= a.sc.dec[2];
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
      const T hv[3] = {Fs0 * T(0.5), Fs1 * T(0.5), Fs2 * T(0.5)};
      const T Nt[3][3] = {{m[4], m[7], m[8]}, {m[7], m[5], m[9]}, {m[8], m[9], m[6]}};
      T g[27];
      full_populations<T>(m[0], uv, hv, Nt, omm, g);
      static_for<Q>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        if constexpr (q == QREST)
          rest_new = g[q];
        else
          put(qc, g[q]);
      });
    } else {
      const PostColl<T> P = post_collision<T>(m[0], m[1], m[2], m[3], m[4], m[5], m[6], m[7], m[8], m[9], Fs0, Fs1,
                                              Fs2, T(0.5), omm);
      static_for<Q>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        if constexpr (q == QREST) {
          rest_new = P.q0;
        } else if constexpr (q < L::opp(q)) {
          T fq, fo;
          pop_pair<L, q, T>(P, fq, fo);
          put(qc, fq);
          put(std::integral_constant<int, L::opp(q)>{}, fo);
        }
      });
    }
    if constexpr (MASK) msk[g2 / GS2 + me] = e.solid ? 1 : 0;
    sol_new = e.solid;
    __syncwarp();
    if (lane == 0) arrive(&staged[row]);
    return true;
  };

  T red[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
  SiteExtra<T, 0> ex;

  if (me == 0) {
    abort_flag = 0;
    for (int s = 0; s < kRawStages; ++s) {
      mbar_init(&full[s], 1);
      rawcnt[s] = 0;
    }
  }
  if (lane == 0) {
    // consumers of row r's ring slots: the output rows among r - 1, r, r + 1
    const int cons = (row - 1 >= 1 ? 1 : 0) + (row >= 1 && row <= BY ? 1 : 0) + (row + 1 <= BY ? 1 : 0);
    mbar_init(&staged[row], 1);
    mbar_init(&done[row], uint32_t(cons));
  }
  if (me == 0) fence_mbar_init();
  if constexpr (MASK) {
    for (int i = me; i < kRowsPad; i += FwdTile<BY>::THREADS) {
      msk[-kRowsPad + i] = 0;
      msk[3 * SITES + i] = 0;
    }
  }
  __syncthreads();
  if (me == 0) {
    prefetch_tensormap(&tmap);
    for (int p = pbase; p < pbase + kRawStages; ++p) issue(p);
  }

  // prologue: planes z0 - 1 and z0 go to fresh ring slots
  load_extra(z0 - 1, ex);
  bool ok = stage(std::integral_constant<int, 0>{}, z0 - 1, g2m, ex);
  up_m1 = up_new;
  sol_m1 = sol_new;
  load_extra(z0, ex);
  ok = ok && stage(std::integral_constant<int, 1>{}, z0, g20, ex);
  up_0 = up_new;
  dn_0 = dn_new;
  rest_0 = rest_new;
  sol_0 = sol_new;
  Fown[0] = Fnext[0];
  Fown[1] = Fnext[1];
  Fown[2] = Fnext[2];
  load_extra(z0 + 1, ex);

  auto iteration = [&](auto par_c, int z) -> bool {
    constexpr int PAR = decltype(par_c)::value;
    if (!stage(std::integral_constant<int, PAR>{}, z + 1, g2p, ex)) return false;
    load_extra(z + 2, ex);
    if (out_row) {
      const uint32_t ph = uint32_t(z + 1 - pbase) & 1u;
      if (!wait_bar(&staged[row - 1], ph) || !wait_bar(&staged[row], ph) || !wait_bar(&staged[row + 1], ph))
        return false;
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
          constexpr int off = D::gidx(q) * SITES - cy * 32 - cx;
          T v = (g == 0 ? P0 : (g == 1 ? P1 : P2))[off];
          if constexpr (W) {
            const uint8_t* mk = cz > 0 ? MM : (cz < 0 ? MP : M0);
            if (mk[-cy * 32 - cx]) {
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
      if constexpr (MASK) {
        if (walls)
          A = gather(std::true_type{});
        else
          A = gather(std::false_type{});
      } else {
        A = gather(std::false_type{});
      }
      // the ring rows r-1, r, r+1 of this plane have been read
      __syncwarp();
      if (lane == 0) {
        arrive(&done[row - 1]);
        arrive(&done[row]);
        arrive(&done[row + 1]);
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
      if (outcol && !sol_0) {
        const long long zc = (long long)z * plane + col;
        LBF_CHECK(a.flags, z >= 0 && z < a.nz && col >= 0 && col < plane && zc + 9 * N < 10 * N);
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
    const int g2t = g2m;
    g2m = g20;
    g20 = g2p;
    g2p = g2t;
    return true;
  };

  if (ok) {
    for (int z = z0; z < z1; z += 2) {
      if (!iteration(std::integral_constant<int, 0>{}, z)) break;
      if (z + 1 < z1 && !iteration(std::integral_constant<int, 1>{}, z + 1)) break;
    }
  }

  // after an abort, loads still in flight land before the CTA exits (bounded): every lane that
  // issued a load waits for the newest plane it issued (the refill two planes later is issued,
  // and waited for, by another lane only once every row has read it). Without an abort every
  // issued plane was read, so nothing is in flight.
  __syncthreads();
  if (abort_flag && lane == 0 && issued >= pbase) {
    const int s = (issued - pbase) % kRawStages;
    mbar_wait_bounded(&full[s], uint32_t((issued - pbase) / kRawStages) & 1u, kWaitPolls);
  }
  __syncthreads();

  if (a.partials != nullptr) {
    double* red_s = reinterpret_cast<double*>(sbase + RAW_BYTES);
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
      a.partials[cta * 8 + me] = s;
    }
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (me == 0) last = atomicAdd(a.counter, 1u) == (unsigned)(nb - 1);
    __syncthreads();
    if (last) {
      __threadfence();
      constexpr int NT = FwdTile<BY>::THREADS;
      double* tree = reinterpret_cast<double*>(sbase);
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
