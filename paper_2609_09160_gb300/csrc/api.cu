// Host side of the C ABI declared in include/lbf.h: parameter validation, workspace layout,
// context state, stream-ordered launches and host <-> device staging.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lbf.h"
#ifdef LBF_DEBUG
#include "../../include/lbf_debug.h"
#endif
#include "aux_kernels.cuh"
#include "dispatch.cuh"

using namespace lbf;

namespace {

thread_local std::string g_last_error;

lbf_status fail(lbf_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

#define LBF_CUDA(call)                                                                        \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail(LBF_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));             \
  } while (0)

constexpr size_t kAlign = 256;
constexpr size_t kStagingMax = size_t(16) << 20;
// 16-bit storage: each group g is multiplied by 2^s_g so that the larger of 16x its initial
// maximum and a physical bound (|p*| = |rho - 1| <= 0.1, |u| <= 0.4 (the stability guard),
// |a2 - u u| <= 0.05) maps to at most 2^15 (FP16 overflows above 65504). Within that range FP16
// keeps its 11-bit significand down to 2^-14 / 2^s, so the floors cost no precision.
constexpr double kTarget16 = 32768.0;
constexpr double kFloor16[3] = {0.1, 0.4, 0.05};

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

size_t storage_bytes(int storage) {
  switch (storage) {
    case LBF_F64: return 8;
    case LBF_F32: return 4;
    case LBF_F16:
    case LBF_BF16: return 2;
  }
  return 0;
}

size_t compute_bytes(int storage) { return storage == LBF_F64 ? 8 : 4; }

struct Layout {
  size_t state[2], mom, mask, phi[2], F[2], G, gphi, partials, scal, staging, total;
  long long npartials;
  size_t staging_bytes;
};

lbf_status check_params(const lbf_params* p) {
  if (p == nullptr) return fail(LBF_EINVAL, "params is NULL");
  if (p->lattice != LBF_D3Q19 && p->lattice != LBF_D3Q27 && p->lattice != LBF_D3Q27H)
    return fail(LBF_EINVAL, "lattice must be LBF_D3Q19, LBF_D3Q27 or LBF_D3Q27H");
  if (p->lattice == LBF_D3Q27H && p->populations)
    return fail(LBF_ENOTSUP, "the population representation collides at second order (D3Q19, D3Q27)");
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return fail(LBF_EINVAL, "nx, ny, nz must be >= 1");
  const double n = double(p->nx) * double(p->ny) * double(p->nz);
  if (n > 4.0e10) return fail(LBF_EINVAL, "lattice too large");
  if (storage_bytes(p->storage) == 0) return fail(LBF_EINVAL, "storage must be LBF_F64, LBF_F32, LBF_F16 or LBF_BF16");
  if (p->rounding != LBF_ROUND_STOCHASTIC && p->rounding != LBF_ROUND_NEAREST)
    return fail(LBF_EINVAL, "rounding must be LBF_ROUND_STOCHASTIC or LBF_ROUND_NEAREST");
  if (p->populations && (p->storage == LBF_F16 || p->storage == LBF_BF16))
    return fail(LBF_ENOTSUP, "the population representation needs LBF_F32 or LBF_F64 storage");
  if (p->populations && p->two_component)
    return fail(LBF_ENOTSUP, "the population representation is single-component only");
  if (p->populations && (p->ny > 65535 || p->nz > 65535))
    return fail(LBF_ENOTSUP, "the population representation launches one block row per (y, z): ny, nz <= 65535");
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(p->force[a]) || !std::isfinite(p->body_accel[a]))
      return fail(LBF_EINVAL, "force and body_accel must be finite");
  if (p->two_component) {
    if (!(p->tau_l > 0.5) || !(p->tau_h > 0.5)) return fail(LBF_EINVAL, "tau_l and tau_h must be > 0.5");
    if (!(p->rho_l > 0.0) || !(p->rho_h > 0.0)) return fail(LBF_EINVAL, "rho_l and rho_h must be > 0");
    const bool wide = p->storage == LBF_F64 || p->storage == LBF_F32;
    if (p->rho_l != p->rho_h && !wide)
      return fail(LBF_ENOTSUP, "two-component with a density contrast needs LBF_F32 or LBF_F64 storage");
    if (p->mask != nullptr && !wide)
      return fail(LBF_ENOTSUP, "two-component with walls needs LBF_F32 or LBF_F64 storage");
    if (!(p->width > 0.0) || !(p->sigma >= 0.0) || !(p->diffusivity >= 0.0))
      return fail(LBF_EINVAL, "need width > 0, sigma >= 0, diffusivity >= 0");
    if (p->force_field != nullptr) return fail(LBF_ENOTSUP, "two-component with a force field is not built");
  } else {
    if (!(p->tau > 0.5) || !std::isfinite(p->tau)) return fail(LBF_EINVAL, "tau must be > 0.5");
    for (int a = 0; a < 3; ++a)
      if (p->body_accel[a] != 0.0)
        return fail(LBF_EINVAL, "body_accel is a two-component parameter (use force for a single component)");
  }
  return LBF_OK;
}

bool has_contrast(const lbf_params* p) { return p->two_component && p->rho_l != p->rho_h; }

int grid_x(int nx, int xout = FwdTile<8>::XOUT) { return (nx + xout - 1) / xout; }
int grid_y(int ny, int by) { return (ny + by - 1) / by; }
int fwd_by(int lattice, int storage, bool mask, bool two) {
  return fwd_rows_lattice(lattice == LBF_D3Q19 ? 19 : 27, int(storage_bytes(storage)), mask, two,
                          lattice == LBF_D3Q27H);
}
int min_zchunk(int nz) { return std::min(8, nz); }
// output rows of the line-aligned kernel for these parameters (0 when it is not built for them)
int aligned_by(const lbf_params* p) {
  if (p->two_component || p->populations || p->storage == LBF_F64) return 0;
  return al_rows(p->lattice == LBF_D3Q19 ? 19 : 27, int(storage_bytes(p->storage)), p->mask != nullptr,
                 p->lattice == LBF_D3Q27H);
}

bool make_layout(const lbf_params* p, Layout* L) {
  if (check_params(p) != LBF_OK) return false;
  const long long N = (long long)p->nx * p->ny * p->nz;
  const size_t sb = storage_bytes(p->storage), cb = compute_bytes(p->storage);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align_up(off + bytes);
    return at;
  };
  // state buffers: 10 moment fields, or Q population fields in the population representation
  // (which also keeps one 10-field moment buffer: read-out target and the solid sites' moments)
  const long long fields = p->populations ? p->lattice : 10;
  L->state[0] = take(fields * N * sb);
  L->state[1] = take(fields * N * sb);
  L->mom = p->populations ? take(10 * N * sb) : 0;
  L->mask = p->mask ? take(N) : 0;
  if (p->two_component) {
    L->phi[0] = take(N * cb);
    L->phi[1] = take(N * cb);
    L->F[0] = take(3 * N * cb);
    L->F[1] = take(3 * N * cb);
    L->G = take(3 * N * cb);
    L->gphi = has_contrast(p) ? take(3 * N * cb) : 0;
  } else {
    L->phi[0] = L->phi[1] = L->F[0] = L->F[1] = L->G = L->gphi = 0;
  }
  const long long gz = (p->nz + min_zchunk(p->nz) - 1) / min_zchunk(p->nz);
  // per-block partial sums of the largest grid either forward kernel can launch
  long long tiles = (long long)grid_x(p->nx) * grid_y(p->ny, fwd_by(p->lattice, p->storage, p->mask != nullptr, p->two_component != 0));
  if (const int aby = aligned_by(p)) tiles = std::max(tiles, (long long)grid_x(p->nx, 32) * grid_y(p->ny, aby));
  // walls: the step may be split into two launches over row ranges (clean rows, rows near walls)
  L->npartials = std::max<long long>(tiles * gz * (p->mask != nullptr ? 2 : 1), 1024);
  L->partials = take(size_t(L->npartials) * 8 * sizeof(double));
  L->scal = take(64 * sizeof(double));
  L->staging_bytes = std::min<size_t>(kStagingMax, size_t(11) * 8 * size_t(N));
  L->staging = take(L->staging_bytes);
  L->total = off;
  return true;
}

float pow2f(int s) { return std::ldexp(1.0f, s); }

int choose_shift(double maxabs, int group, bool hinted) {
  double m = maxabs > 0.0 && std::isfinite(maxabs) ? maxabs : 0.0;
  if (!hinted) m = std::max(16.0 * m, kFloor16[group]);
  if (!(m > 0.0)) m = kFloor16[group];
  int s = (int)std::floor(std::log2(kTarget16 / m));
  return std::max(-30, std::min(60, s));
}

}  // namespace

struct lbf_ctx {
  lbf_params prm;
  Layout lay;
  int Q, storage;
  bool has_mask, two;
  int nx, ny, nz;
  long long N;
  unsigned char* ws;
  void* state[2];
  int cur;
  uint8_t* mask_d;
  void* phi[2];
  void* F[2];
  void* G;
  void* gphi;      // density contrast: grad phi of the newest phase field
  bool contrast;   // two components with rho_l != rho_h
  int pcur;
  double* partials;
  double* sums;       // 8 doubles at scal
  unsigned* flags;    // after sums
  unsigned* absmax;   // 3 words
  unsigned* counter;  // blocks done in the fused reduction
  unsigned char* staging;
  Scales sc;
  cudaStream_t stream;
  int zchunk;
  dim3 fgrid, agrid;
  KernelInfo fwd, adj;
  KernelInfo fwd_direct;  // the same step loading every site directly (sources TMA cannot read)
  KernelInfo fwd_tma30;   // the 30-column TMA kernel (buffers the aligned kernel cannot address)
  bool tma;             // the forward kernel stages plane patches with TMA
  bool aligned;         // the forward kernel is the line-aligned one (TMA loads and stores)
  CUtensorMap tmap[2];  // tensor maps of the two state buffers (TMA source)
  CUtensorMap smap[2];  // tensor maps of the two state buffers (TMA store destination)
  bool sums_valid;
  bool unstable_seen;
  double omega, nu_l, nu_h;
  unsigned long long steps_done;  // forward launches so far: selects the rounding words of a step
  bool pops;                      // population representation (state buffers hold Q fields)
  PopKernels popk;
  void* mom;                      // pops: internal moment state (read-out target, solid sites kept)
  dim3 pop_grid;                  // pops: (ceil(nx / 256), ny, nz) blocks of 256 threads
  // walls confined to a band of rows: the rows clear of every solid site and of its neighbours
  // ("clean") run the periodic line-aligned kernel, the others the masked 30-column kernel on a
  // side stream; the last block of either launch adds both launches' partial sums
  bool split;
  int clean_begin, clean_rows, dirty_begin, dirty_rows;
  KernelInfo fwd_clean;
  dim3 grid_clean, grid_dirty;
  int zchunk_clean, zchunk_dirty;
  CUtensorMap tmap_clean[2];
  cudaStream_t side;
  cudaEvent_t ev_fork, ev_join;
};

namespace {

KernelInfo forward_for(int Q, int storage, bool mask, int two, bool field, bool tma, bool nearest) {
  return forward_kernel_for(Q, storage, mask, two, field, tma, nearest);
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// TMA is used when a row of the state is a whole number of 16-byte units (the tensor map needs
// 16-byte strides) and the driver provides the encoder
bool tma_eligible(int storage, int nx) {
  return (size_t(nx) * storage_bytes(storage)) % 16 == 0 && tensor_map_encoder() != nullptr &&
         std::getenv("LBF_NO_TMA") == nullptr;
}

// 4-D map over a state buffer: dims (x, y, z, field), box (box_x, box_y, 1, 10)
lbf_status encode_state_map(const lbf_ctx* c, const void* base, CUtensorMap* out, int box_x, int box_y);
KernelInfo adjoint_for(int Q, int storage, bool mask) { return adjoint_kernel_for(Q, storage, mask); }

lbf_status prepare(const KernelInfo& k) {
  if (k.fn == nullptr) return LBF_OK;
  LBF_CUDA(cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem));
  // all of the unified L1/shared storage as shared memory: the rings decide how many CTAs fit
  LBF_CUDA(cudaFuncSetAttribute(k.fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  return LBF_OK;
}

bool is_device_pointer(const void* p) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

// device address of page-locked host memory (mapped into the device's address space), or null for
// pageable host memory: kernels read and write pinned buffers directly over the host link
const void* mapped_host_pointer(const void* p) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return attr.type == cudaMemoryTypeHost ? attr.devicePointer : nullptr;
}

unsigned blocks_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  return (unsigned)std::max<long long>(1, std::min<long long>(b, 65535LL * 16));
}

template <class Tin, class S>
void launch_encode(const void* src, long long stride, long long site0, long long count, void* dst, long long N, Scales sc,
                   cudaStream_t st) {
  k_encode<Tin, S><<<blocks_for(count, 256), 256, 0, st>>>(static_cast<const Tin*>(src), stride, site0, count,
                                                           static_cast<S*>(dst), N, sc);
}

template <class Tin>
void encode_dispatch(int storage, const void* src, long long stride, long long site0, long long count, void* dst,
                     long long N, Scales sc, cudaStream_t st) {
  switch (storage) {
    case LBF_F64: launch_encode<Tin, double>(src, stride, site0, count, dst, N, sc, st); break;
    case LBF_F32: launch_encode<Tin, float>(src, stride, site0, count, dst, N, sc, st); break;
    case LBF_F16: launch_encode<Tin, __half>(src, stride, site0, count, dst, N, sc, st); break;
    case LBF_BF16: launch_encode<Tin, __nv_bfloat16>(src, stride, site0, count, dst, N, sc, st); break;
  }
}

template <class S, class Tout>
void launch_decode(const void* src, long long N, long long site0, long long count, void* dst, long long stride, Scales sc,
                   cudaStream_t st) {
  k_decode<S, Tout><<<blocks_for(count, 256), 256, 0, st>>>(static_cast<const S*>(src), N, site0, count,
                                                            static_cast<Tout*>(dst), stride, sc);
}

template <class Tout>
void decode_dispatch(int storage, const void* src, long long N, long long site0, long long count, void* dst,
                     long long stride, Scales sc, cudaStream_t st) {
  switch (storage) {
    case LBF_F64: launch_decode<double, Tout>(src, N, site0, count, dst, stride, sc, st); break;
    case LBF_F32: launch_decode<float, Tout>(src, N, site0, count, dst, stride, sc, st); break;
    case LBF_F16: launch_decode<__half, Tout>(src, N, site0, count, dst, stride, sc, st); break;
    case LBF_BF16: launch_decode<__nv_bfloat16, Tout>(src, N, site0, count, dst, stride, sc, st); break;
  }
}

template <class Tin, class Tout>
__global__ void k_convert(const Tin* __restrict__ a, Tout* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = static_cast<Tout>(a[i]);
}

void convert(const void* a, int da, void* b, int db, long long n, cudaStream_t st) {
  const unsigned g = blocks_for(n, 256);
  if (da == LBF_F64 && db == LBF_F64) k_convert<double, double><<<g, 256, 0, st>>>((const double*)a, (double*)b, n);
  else if (da == LBF_F64) k_convert<double, float><<<g, 256, 0, st>>>((const double*)a, (float*)b, n);
  else if (db == LBF_F64) k_convert<float, double><<<g, 256, 0, st>>>((const float*)a, (double*)b, n);
  else k_convert<float, float><<<g, 256, 0, st>>>((const float*)a, (float*)b, n);
}

PhaseParams phase_params(const lbf_ctx* c) {
  PhaseParams pp;
  pp.nx = c->nx;
  pp.ny = c->ny;
  pp.nz = c->nz;
  pp.N = c->N;
  pp.D = c->prm.diffusivity;
  pp.lambda = 4.0 * c->prm.diffusivity / c->prm.width;
  pp.beta = 12.0 * c->prm.sigma / c->prm.width;
  pp.kappa = 1.5 * c->prm.sigma * c->prm.width;
  for (int a = 0; a < 3; ++a) {
    pp.body[a] = c->prm.force[a];
    pp.accel[a] = c->prm.body_accel[a];
  }
  pp.rho_l = c->prm.rho_l;
  pp.drho = c->prm.rho_h - c->prm.rho_l;
  pp.mask = c->mask_d;
  pp.sc = c->sc;
  pp.zchunk = c->zchunk;
  return pp;
}

// phase-field kernels: the fused step's x-y tiles (30 x kPhaseRows outputs), z-chunks of zchunk
dim3 phase_block() { return dim3(32, kPhaseRows + 2, 1); }
dim3 phase_grid(const lbf_ctx* c) {
  return dim3((c->nx + 29) / 30, (c->ny + kPhaseRows - 1) / kPhaseRows, (c->nz + c->zchunk - 1) / c->zchunk);
}

template <class T>
void launch_forces_T(lbf_ctx* c, int which) {
  k_phase_forces<T><<<phase_grid(c), phase_block(), 0, c->stream>>>(
      static_cast<const T*>(c->phi[which]), static_cast<T*>(c->F[which]), static_cast<T*>(c->G),
      c->contrast ? static_cast<T*>(c->gphi) : nullptr, phase_params(c));
}

void launch_forces(lbf_ctx* c, int which) {
  if (c->storage == LBF_F64) launch_forces_T<double>(c, which);
  else launch_forces_T<float>(c, which);
}

template <class S, class T>
void launch_advance_T(lbf_ctx* c) {
  k_phase_advance<S, T><<<phase_grid(c), phase_block(), 0, c->stream>>>(
      static_cast<const S*>(c->state[c->cur]), static_cast<const T*>(c->phi[c->pcur]), static_cast<const T*>(c->G),
      static_cast<T*>(c->phi[1 - c->pcur]), phase_params(c));
}

void launch_advance(lbf_ctx* c) {
  switch (c->storage) {
    case LBF_F64: launch_advance_T<double, double>(c); break;
    case LBF_F32: launch_advance_T<float, float>(c); break;
    case LBF_F16: launch_advance_T<__half, float>(c); break;
    case LBF_BF16: launch_advance_T<__nv_bfloat16, float>(c); break;
  }
}

FwdParams forward_params(const lbf_ctx* c, const void* src, void* dst, bool reduce) {
  FwdParams a;
  std::memset(&a, 0, sizeof(a));
  a.src = src;
  a.dst = dst;
  a.mask = c->mask_d;
  a.force_field = c->prm.force_field;
  for (int k = 0; k < 3; ++k) a.force[k] = c->prm.force[k];
  a.omega = c->omega;
  if (c->two) {
    a.phi_old = c->phi[c->pcur];
    a.phi_new = c->phi[1 - c->pcur];
    a.F_old = c->F[c->pcur];
    a.F_new = c->F[1 - c->pcur];
    a.grad_phi = c->gphi;
    a.rho_l = c->prm.rho_l;
    a.rho_h = c->prm.rho_h;
    a.nu_l = c->nu_l;
    a.nu_h = c->nu_h;
  }
  a.nx = c->nx;
  a.ny = c->ny;
  a.nz = c->nz;
  a.N = c->N;
  a.sc = c->sc;
  a.partials = reduce ? c->partials : nullptr;
  a.sums = c->sums;
  a.counter = c->counter;
  a.flags = c->flags;
  a.zchunk = c->zchunk;
  a.umax2 = 0.16f;
  a.salt = fmix32(uint32_t(c->steps_done) * 0x9E3779B9u + 0x7F4A7C15u);
  set_fp32_copies(a);
  return a;
}

PopParams pop_params(const lbf_ctx* c, const void* src, void* dst, bool reduce) {
  PopParams p;
  std::memset(&p, 0, sizeof(p));
  p.src = src;
  p.dst = dst;
  p.mom = c->mom;
  p.mask = c->mask_d;
  p.force_field = c->prm.force_field;
  for (int k = 0; k < 3; ++k) {
    p.force[k] = c->prm.force[k];
    p.force_f[k] = float(c->prm.force[k]);
  }
  p.omega = c->omega;
  p.omega_f = float(c->omega);
  p.nx = c->nx;
  p.ny = c->ny;
  p.nz = c->nz;
  p.N = c->N;
  (void)reduce;  // the population step does not fuse the sums: lbf_reduce takes them from the state
  p.flags = c->flags;
  p.umax2 = 0.16f;
  return p;
}

// population representation: the internal moments of the current state into c->mom
lbf_status pop_moments(lbf_ctx* c) {
  PopParams pp = pop_params(c, c->state[c->cur], nullptr, false);
  void* args[] = {&pp};
  LBF_CUDA(cudaLaunchKernel(c->popk.moments, c->pop_grid, dim3(kPopThreads), args, 0, c->stream));
  return LBF_OK;
}

lbf_status encode_state_map(const lbf_ctx* c, const void* base, CUtensorMap* out, int box_x, int box_y) {
  CUtensorMapDataType dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  switch (c->storage) {
    case LBF_F64: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT64; break;
    case LBF_F32: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT32; break;
    case LBF_F16: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT16; break;
    case LBF_BF16: dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; break;
  }
  const cuuint64_t es = storage_bytes(c->storage);
  const cuuint64_t dims[4] = {cuuint64_t(c->nx), cuuint64_t(c->ny), cuuint64_t(c->nz), 10};
  const cuuint64_t strides[3] = {es * c->nx, es * c->nx * c->ny, es * cuuint64_t(c->N)};
  const cuuint32_t box[4] = {cuuint32_t(box_x), cuuint32_t(box_y), 1, 10};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = tensor_map_encoder()(out, dt, 4, const_cast<void*>(base), dims, strides, box, estr,
                                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(LBF_ECUDA, "cuTensorMapEncodeTiled failed with code " + std::to_string(int(r)));
  return LBF_OK;
}

// z-chunk of a launch of `tiles` x-y tiles: the CTAs of one tile column march through nz / chunks
// planes each, restaging two planes per chunk. Large lattices: the longest chunk (16 to 64 planes)
// that still gives at least kMinWaves waves of resident CTAs, since fewer, longer-lived CTAs start
// and stage in step and overlap their phases worse (D3Q19 FP32: 256^3 best at 24-plane chunks, 6.2
// waves, +3.5% over 37-plane chunks at 3.9 waves; 512^3 best at 64, 18 waves). Lattices too small
// for that: the chunk count that minimises (1 + restaged planes) / (fraction of the last wave busy)
// (the 128^3 droplet: 15-plane chunks, 1.9 waves, 15.6 GLUPS against 14.7 at 8 planes).
constexpr double kMinWaves = 6.0;
int choose_zchunk(int nz, long long tiles, double resident) {
  for (int chunks = 1; chunks <= nz; ++chunks) {
    const int z = (nz + chunks - 1) / chunks;
    if (z < std::max(16, min_zchunk(nz))) break;
    const long long nchunks = (nz + z - 1) / z;
    if (z <= 64 && double(tiles * nchunks) / resident >= kMinWaves) return z;
  }
  int zc = nz;
  double best = 1e30;
  for (int chunks = 1; chunks <= nz; ++chunks) {
    const int z = (nz + chunks - 1) / chunks;
    if (z < min_zchunk(nz)) break;
    if (z > 64) continue;  // long chunks leave too few CTAs to overlap their pipelines
    const long long nchunks = (nz + z - 1) / z;
    const double waves = double(tiles * nchunks) / resident;
    const double busy = waves / std::ceil(waves);
    const double cost = (1.0 + 2.0 / z) / busy;
    if (cost < best - 1e-9) {
      best = cost;
      zc = z;
    }
  }
  return std::min(zc, nz);
}

#ifndef LBF_SPLIT_ZCHUNK
#define LBF_SPLIT_ZCHUNK 32
#endif

// Row split for walls that occupy few rows (a channel's walls): row y is clean when rows y-1, y,
// y+1 (periodic) hold no solid site at any x and z, so every population its outputs pull comes
// from a fluid site and the periodic kernel (no mask logic) computes them exactly. When the clean
// rows form one cyclic run of at least half the rows, that run goes to the line-aligned periodic
// kernel and the remaining rows to the masked kernel. Only where the aligned kernel is the one
// the library picks for periodic lattices of this size and type.
lbf_status setup_split(lbf_ctx* c, const lbf_params* p, const Layout& L, int sms, bool nearest,
                       const std::string& kname) {
  if (!c->has_mask || c->two || c->pops || !c->tma || c->aligned || p->force_field != nullptr || LBF_AL_TMA_STORE ||
      kname == "cta" || kname == "aligned")
    return LBF_OK;
  const long long plane_sites = (long long)c->nx * c->ny;
  const bool q19_f32 = c->Q == LBF_D3Q19 && c->storage == LBF_F32;
  const bool forced = kname == "split";  // LBF_KERNEL=split: any plane size (tests)
  if ((!forced && plane_sites < (q19_f32 ? 256LL * 256LL : 512LL * 512LL)) ||
      !((c->Q == LBF_D3Q19 && c->storage != LBF_F64) || (c->Q == LBF_D3Q27 && c->storage == LBF_F32)))
    return LBF_OK;
  const KernelInfo al = aligned_kernel_for(c->Q, c->storage, false, false, nearest);
  if (al.fn == nullptr) return LBF_OK;
  const int nx = c->nx, ny = c->ny, nz = c->nz;
  std::vector<char> solid_row(ny, 0);
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y) {
      if (solid_row[y]) continue;
      const uint8_t* row = p->mask + ((long long)z * ny + y) * nx;
      for (int x = 0; x < nx; ++x)
        if (row[x] != 0) {
          solid_row[y] = 1;
          break;
        }
    }
  std::vector<char> clean(ny);
  int nclean = 0;
  for (int y = 0; y < ny; ++y) {
    clean[y] = !(solid_row[(y + ny - 1) % ny] || solid_row[y] || solid_row[(y + 1) % ny]);
    nclean += clean[y];
  }
  if (nclean == ny || nclean < ny / 2) return LBF_OK;  // no solid site at all, or walls everywhere
  // the longest cyclic run of clean rows starts right after a row that is not clean
  int best_begin = 0, best_len = 0;
  for (int y = 0; y < ny; ++y) {
    if (!clean[y] || clean[(y + ny - 1) % ny]) continue;
    int len = 0;
    while (len < ny && clean[(y + len) % ny]) ++len;
    if (len > best_len) best_len = len, best_begin = y;
  }
  // whole tiles on both sides where possible: the clean run shrinks to a multiple of the aligned
  // tile height such that the rows left to the masked kernel fill whole tiles of its own height
  for (int len = best_len / al.by * al.by; len >= 2 * al.by && len >= ny / 2; len -= al.by)
    if ((ny - len) % c->fwd.by == 0) {
      best_len = len;
      break;
    }
  if (best_len < ny / 2 || best_len < 2 * al.by) return LBF_OK;
  lbf_status st;
  if ((st = prepare(al)) != LBF_OK) return st;
  int per_sm_al = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_al, al.fn, al.threads, al.smem) != cudaSuccess)
    return fail(LBF_ECUDA, std::string("device query failed: ") + cudaGetErrorString(cudaGetLastError()));
  const int dirty_rows = ny - best_len;
  const long long tiles_clean = (long long)grid_x(nx, al.xout) * grid_y(best_len, al.by);
  const long long tiles_dirty = (long long)grid_x(nx, c->fwd.xout) * grid_y(dirty_rows, c->fwd.by);
  int zcc = choose_zchunk(nz, tiles_clean, double(sms) * std::max(per_sm_al, 1));
  if (const char* e = std::getenv("LBF_ZCHUNK")) {  // the same override as for a single launch
    const int v = std::atoi(e);
    if (v >= 1) zcc = std::min(nz, std::max(min_zchunk(nz), v));
  }
  // the rows near walls run beside the clean launch on a few CTAs (tuning define LBF_SPLIT_ZCHUNK)
  const int zcd = std::min(LBF_SPLIT_ZCHUNK, nz);
  const dim3 gc(grid_x(nx, al.xout), grid_y(best_len, al.by), (nz + zcc - 1) / zcc);
  const dim3 gd(grid_x(nx, c->fwd.xout), grid_y(dirty_rows, c->fwd.by), (nz + zcd - 1) / zcd);
  const long long blocks = (long long)gc.x * gc.y * gc.z + (long long)gd.x * gd.y * gd.z;
  if (blocks > L.npartials) return LBF_OK;
  for (int k = 0; k < 2; ++k)
    if ((st = encode_state_map(c, c->state[k], &c->tmap_clean[k], al.box_x, al.by + 2)) != LBF_OK) return st;
  int lo = 0, hi = 0;
  LBF_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
  LBF_CUDA(cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, hi));  // dispatched first
  LBF_CUDA(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
  LBF_CUDA(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
  c->fwd_clean = al;
  c->clean_begin = best_begin;
  c->clean_rows = best_len;
  c->dirty_begin = (best_begin + best_len) % ny;
  c->dirty_rows = dirty_rows;
  c->zchunk_clean = zcc;
  c->zchunk_dirty = zcd;
  c->grid_clean = gc;
  c->grid_dirty = gd;
  c->split = true;
  return LBF_OK;
}

// one step as two launches over row ranges: the rows near walls (masked kernel) on the side stream,
// the clean rows (periodic line-aligned kernel) on the context's stream, joined at the end of the
// step; the two launches share the block counter, and the last block of either adds all partials
lbf_status launch_split(lbf_ctx* c, const FwdParams& a, int ks) {
  FwdParams ad = a, ac = a;
  const long long nd = (long long)c->grid_dirty.x * c->grid_dirty.y * c->grid_dirty.z;
  const long long nc = (long long)c->grid_clean.x * c->grid_clean.y * c->grid_clean.z;
  ad.y_begin = c->dirty_begin;
  ad.y_rows = c->dirty_rows;
  ad.zchunk = c->zchunk_dirty;
  ad.block_base = 0;
  ad.final_blocks = nd + nc;
  ac.y_begin = c->clean_begin;
  ac.y_rows = c->clean_rows;
  ac.zchunk = c->zchunk_clean;
  ac.block_base = nd;
  ac.final_blocks = nd + nc;
  ac.mask = nullptr;  // every site of the clean rows and of their neighbour rows is fluid
  CUtensorMap tmd = c->tmap[ks], tmc = c->tmap_clean[ks], none;
  std::memset(&none, 0, sizeof(none));
  LBF_CUDA(cudaEventRecord(c->ev_fork, c->stream));
  LBF_CUDA(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
  void* argd[] = {&ad, &tmd, &none};
  LBF_CUDA(cudaLaunchKernel(c->fwd.fn, c->grid_dirty, dim3(32, c->fwd.threads / 32, 1), argd, c->fwd.smem, c->side));
  LBF_CUDA(cudaEventRecord(c->ev_join, c->side));
  void* argc[] = {&ac, &tmc, &none};
  LBF_CUDA(cudaLaunchKernel(c->fwd_clean.fn, c->grid_clean, dim3(32, c->fwd_clean.threads / 32, 1), argc,
                            c->fwd_clean.smem, c->stream));
  LBF_CUDA(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
  return LBF_OK;
}

lbf_status launch_forward(lbf_ctx* c, const void* src, void* dst, bool reduce) {
  if (c->pops) {
    PopParams pp = pop_params(c, src, dst, reduce);
    void* args[] = {&pp};
    LBF_CUDA(cudaLaunchKernel(c->popk.step, c->pop_grid, dim3(kPopThreads), args, 0, c->stream));
    return LBF_OK;
  }
  FwdParams a = forward_params(c, src, dst, reduce);
  ++c->steps_done;
  if (c->split) {
    const int ks = src == c->state[0] ? 0 : (src == c->state[1] ? 1 : -1);
    const int kd = dst == c->state[0] ? 0 : (dst == c->state[1] ? 1 : -1);
    if (ks >= 0 && kd >= 0) return launch_split(c, a, ks);
  }
  CUtensorMap tm, sm;
  std::memset(&tm, 0, sizeof(tm));
  std::memset(&sm, 0, sizeof(sm));
  const KernelInfo* k = &c->fwd;
  const bool aligned16 = reinterpret_cast<uintptr_t>(src) % 16 == 0;  // a tensor map needs a 16-byte base
  if (c->aligned) {
    const int ks = src == c->state[0] ? 0 : (src == c->state[1] ? 1 : -1);
    const int kd = dst == c->state[0] ? 0 : (dst == c->state[1] ? 1 : -1);
    if (ks >= 0 && kd >= 0) {
      tm = c->tmap[ks];
      sm = c->smap[kd];
    } else if (aligned16 && reinterpret_cast<uintptr_t>(dst) % 16 == 0) {
      lbf_status st = encode_state_map(c, src, &tm, c->fwd.box_x, c->fwd.by + 2);
      if (st == LBF_OK) st = encode_state_map(c, dst, &sm, 32, c->fwd.by);
      if (st != LBF_OK) return st;
    } else if (aligned16) {  // dst cannot take TMA stores: 30-column kernel with TMA loads
      k = &c->fwd_tma30;
      lbf_status st = encode_state_map(c, src, &tm, k->box_x, k->by + 2);
      if (st != LBF_OK) return st;
    } else {
      k = &c->fwd_direct;
    }
  } else if (c->tma) {
    const int box_y = k->by + 2;
    if (src == c->state[0]) {
      tm = c->tmap[0];
    } else if (src == c->state[1]) {
      tm = c->tmap[1];
    } else if (!aligned16) {
      k = &c->fwd_direct;
    } else {
      lbf_status st = encode_state_map(c, src, &tm, k->box_x, box_y);
      if (st != LBF_OK) return st;
    }
  }
  void* args[] = {&a, &tm, &sm};
  const dim3 grid(grid_x(c->nx, k->xout), grid_y(c->ny, k->by), c->fgrid.z);
  LBF_CUDA(cudaLaunchKernel(k->fn, grid, dim3(32, k->threads / 32, 1), args, k->smem, c->stream));
  return LBF_OK;
}

lbf_status finalize_sums(lbf_ctx* c, long long nblocks) {
  k_reduce_final<<<1, 256, 0, c->stream>>>(c->partials, nblocks, c->sums);
  LBF_CUDA(cudaGetLastError());
  c->sums_valid = true;
  return LBF_OK;
}

template <class S>
void launch_reduce_state_T(lbf_ctx* c, unsigned grid) {
  const void* st = c->pops ? c->mom : c->state[c->cur];
  k_reduce_state<S><<<grid, 256, 0, c->stream>>>(static_cast<const S*>(st), c->N, c->mask_d,
                                                   c->two ? c->phi[c->pcur] : nullptr, c->storage == LBF_F64, c->sc,
                                                   c->partials);
}

lbf_status reduce_state(lbf_ctx* c) {
  if (c->pops) {
    const lbf_status st = pop_moments(c);
    if (st != LBF_OK) return st;
  }
  const unsigned grid = (unsigned)std::min<long long>(1024, std::max<long long>(1, (c->N + 255) / 256));
  switch (c->storage) {
    case LBF_F64: launch_reduce_state_T<double>(c, grid); break;
    case LBF_F32: launch_reduce_state_T<float>(c, grid); break;
    case LBF_F16: launch_reduce_state_T<__half>(c, grid); break;
    case LBF_BF16: launch_reduce_state_T<__nv_bfloat16>(c, grid); break;
  }
  LBF_CUDA(cudaGetLastError());
  return finalize_sums(c, grid);
}

void set_scales(lbf_ctx* c, const double m[3]) {
  for (int g = 0; g < 3; ++g) {
    if (c->storage == LBF_F16 || c->storage == LBF_BF16) {
      const double hint = c->prm.scale_hint[g];
      const int s = hint > 0.0 ? choose_shift(hint, g, true) : choose_shift(m[g], g, false);
      c->sc.enc[g] = pow2f(s);
      c->sc.dec[g] = pow2f(-s);
    } else {
      c->sc.enc[g] = 1.0f;
      c->sc.dec[g] = 1.0f;
    }
  }
}

template <class T>
void host_absmax(const T* src, long long N, double m[3]) {
  m[0] = m[1] = m[2] = 0.0;
  for (long long i = 0; i < N; ++i) {
    const double p = src[i], ux = src[N + i], uy = src[2 * N + i], uz = src[3 * N + i];
    m[0] = std::max(m[0], std::fabs(p));
    m[1] = std::max(m[1], std::max(std::fabs(ux), std::max(std::fabs(uy), std::fabs(uz))));
    const double n[6] = {src[4 * N + i] - ux * ux, src[5 * N + i] - uy * uy, src[6 * N + i] - uz * uz,
                         src[7 * N + i] - ux * uy, src[8 * N + i] - ux * uz, src[9 * N + i] - uy * uz};
    for (int k = 0; k < 6; ++k) m[2] = std::max(m[2], std::fabs(n[k]));
  }
}

#ifdef LBF_DEBUG
// one CTA waits, with the fused step's bounded wait, on an mbarrier that nothing arrives on (no
// copy is ever issued), and reports the give-up through the fused step's error bit
__global__ void k_wait_probe(unsigned* flags, uint32_t polls) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0u, polls)) atomicOr(flags, 2u);
}
#endif

}  // namespace

// lets the other translation units of the library report through lbf_last_error()
void lbf_internal_set_last_error(const char* msg) { g_last_error = msg ? msg : ""; }

extern "C" {

int lbf_version(void) { return 1; }

int lbf_kernels_per_step(const lbf_ctx* c) {
  if (c == nullptr) return 0;
  return (c->split ? 2 : 1) + (c->two ? 2 : 0);
}

const char* lbf_last_error(void) { return g_last_error.c_str(); }

const char* lbf_status_string(int s) {
  switch (s) {
    case LBF_OK: return "LBF_OK";
    case LBF_EINVAL: return "LBF_EINVAL";
    case LBF_ENOMEM: return "LBF_ENOMEM";
    case LBF_ECUDA: return "LBF_ECUDA";
    case LBF_EUNSTABLE: return "LBF_EUNSTABLE";
    case LBF_EINTERNAL: return "LBF_EINTERNAL";
    case LBF_ENOTSUP: return "LBF_ENOTSUP";
  }
  return "LBF_UNKNOWN";
}

lbf_status lbf_validate(const lbf_params* params) { return check_params(params); }

size_t lbf_workspace_bytes(const lbf_params* params) {
  Layout L;
  if (!make_layout(params, &L)) return 0;
  return L.total;
}

lbf_status lbf_create(lbf_ctx** out, const lbf_params* params, void* workspace, size_t bytes) {
  if (out == nullptr) return fail(LBF_EINVAL, "out is NULL");
  *out = nullptr;
  lbf_status st = check_params(params);
  if (st != LBF_OK) return st;
  Layout L;
  make_layout(params, &L);
  if (workspace == nullptr) return fail(LBF_EINVAL, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(workspace) % kAlign != 0) return fail(LBF_ENOMEM, "workspace must be 256-byte aligned");
  if (bytes < L.total)
    return fail(LBF_ENOMEM, "workspace too small: need " + std::to_string(L.total) + " bytes");
  lbf_ctx* c = new lbf_ctx();
  c->prm = *params;
  c->prm.mask = nullptr;  // host mask is copied, never kept
  c->lay = L;
  c->Q = params->lattice;
  c->storage = params->storage;
  c->has_mask = params->mask != nullptr;
  c->two = params->two_component != 0;
  c->nx = params->nx;
  c->ny = params->ny;
  c->nz = params->nz;
  c->N = (long long)c->nx * c->ny * c->nz;
  c->ws = static_cast<unsigned char*>(workspace);
  c->state[0] = c->ws + L.state[0];
  c->state[1] = c->ws + L.state[1];
  c->cur = 0;
  c->pops = params->populations != 0;
  c->mom = c->pops ? c->ws + L.mom : nullptr;
  c->pop_grid = dim3((c->nx + kPopThreads - 1) / kPopThreads, c->ny, c->nz);
  c->mask_d = c->has_mask ? reinterpret_cast<uint8_t*>(c->ws + L.mask) : nullptr;
  for (int k = 0; k < 2; ++k) {
    c->phi[k] = c->two ? c->ws + L.phi[k] : nullptr;
    c->F[k] = c->two ? c->ws + L.F[k] : nullptr;
  }
  c->G = c->two ? c->ws + L.G : nullptr;
  c->contrast = has_contrast(params);
  c->gphi = c->contrast ? c->ws + L.gphi : nullptr;
  c->pcur = 0;
  c->partials = reinterpret_cast<double*>(c->ws + L.partials);
  c->sums = reinterpret_cast<double*>(c->ws + L.scal);
  c->flags = reinterpret_cast<unsigned*>(c->sums + 8);
  c->absmax = c->flags + 4;
  c->counter = c->flags + 8;
  c->staging = c->ws + L.staging;
  c->stream = static_cast<cudaStream_t>(params->stream);
  c->omega = 1.0 / params->tau;
  c->nu_l = (params->tau_l - 0.5) / 3.0;
  c->nu_h = (params->tau_h - 0.5) / 3.0;
  c->sums_valid = false;
  c->unstable_seen = false;
  c->steps_done = 0;
  const double m0[3] = {0.0, 0.0, 0.0};
  set_scales(c, m0);

  c->tma = tma_eligible(c->storage, c->nx);
  const bool nearest = params->rounding == LBF_ROUND_NEAREST;
  const int two_mode = c->two ? (c->contrast ? 2 : 1) : 0;
  c->fwd = forward_for(c->Q, c->storage, c->has_mask, two_mode, params->force_field != nullptr, c->tma, nearest);
  c->fwd_tma30 = c->fwd;
  c->aligned = false;
  // single-component TMA steps: the line-aligned kernel where it measured faster than the 30-column
  // one on one GB300: periodic D3Q19 FP32 on planes of at least 256 x 256 sites (8-row tiles: +23%
  // at 512^3, +8% at 256^3), periodic D3Q19 16-bit and D3Q27 FP32 on planes of at least 512 x 512
  // (+3%, +2% at 512^3); slower with walls, for D3Q27h and for 16-bit D3Q27. LBF_KERNEL=aligned or
  // cta forces one of them.
  const char* kind = std::getenv("LBF_KERNEL");
  const std::string kname = kind ? kind : "";
  const long long plane_sites = (long long)c->nx * c->ny;
  const bool q19_f32 = c->Q == LBF_D3Q19 && c->storage == LBF_F32;
  const bool large = plane_sites >= (q19_f32 ? 256LL * 256LL : 512LL * 512LL);
  const bool policy = !c->has_mask && params->force_field == nullptr && large &&
                      ((c->Q == LBF_D3Q19 && c->storage != LBF_F64) || (c->Q == LBF_D3Q27 && c->storage == LBF_F32));
  if (c->tma && !c->two && !c->pops && (kname == "aligned" || (kname.empty() && policy))) {
    const KernelInfo al = aligned_kernel_for(c->Q, c->storage, c->has_mask, params->force_field != nullptr, nearest);
    if (al.fn != nullptr) {
      c->fwd = al;
      c->aligned = true;
    }
  }
  c->popk = c->pops ? pop_kernels_for(c->Q, c->storage, c->has_mask, params->force_field != nullptr)
                    : PopKernels{nullptr, nullptr, nullptr};
  if (c->pops && c->popk.step == nullptr) {
    delete c;
    return fail(LBF_ENOTSUP, "no population kernel for this combination");
  }
  c->fwd_direct = c->tma ? forward_for(c->Q, c->storage, c->has_mask, two_mode, params->force_field != nullptr, false,
                                        params->rounding == LBF_ROUND_NEAREST)
                         : c->fwd;
  c->adj = adjoint_for(c->Q, c->storage, c->has_mask);
  if (c->fwd.fn == nullptr || c->fwd_direct.fn == nullptr) {
    delete c;
    return fail(LBF_ENOTSUP, "no kernel for this combination");
  }
  auto cleanup = [&](lbf_status s) {
    lbf_destroy(c);
    return s;
  };
  if ((st = prepare(c->fwd)) != LBF_OK) return cleanup(st);
  if ((st = prepare(c->fwd_tma30)) != LBF_OK) return cleanup(st);
  if ((st = prepare(c->fwd_direct)) != LBF_OK) return cleanup(st);
  if ((st = prepare(c->adj)) != LBF_OK) return cleanup(st);

  // z-chunk: the CTAs of one (x, y) tile column march through nz / chunks planes each. Choose the
  // chunk count that minimises (1 + restaged planes) / (fraction of the last wave that is busy).
  int dev = 0, sms = 1, per_sm = 1;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, c->fwd.fn, c->fwd.threads, c->fwd.smem) != cudaSuccess)
    return cleanup(fail(LBF_ECUDA, std::string("device query failed: ") + cudaGetErrorString(cudaGetLastError())));
  per_sm = std::max(per_sm, 1);
  const long long tiles = (long long)grid_x(c->nx, c->fwd.xout) * grid_y(c->ny, c->fwd.by);
  int zc = choose_zchunk(c->nz, tiles, double(sms) * per_sm);
  if (const char* e = std::getenv("LBF_ZCHUNK")) {
    const int v = std::atoi(e);
    if (v >= 1) zc = std::max(min_zchunk(c->nz), v);
  }
  c->zchunk = std::min(zc, c->nz);
  c->fgrid = dim3(grid_x(c->nx, c->fwd.xout), grid_y(c->ny, c->fwd.by), (c->nz + c->zchunk - 1) / c->zchunk);
  c->agrid = c->adj.fn ? dim3(grid_x(c->nx), grid_y(c->ny, c->adj.by), (c->nz + c->zchunk - 1) / c->zchunk) : dim3(1, 1, 1);
  if (c->tma) {
    for (int k = 0; k < 2; ++k) {
      if ((st = encode_state_map(c, c->state[k], &c->tmap[k], c->fwd.box_x, c->fwd.by + 2)) != LBF_OK) return cleanup(st);
      if (c->aligned && (st = encode_state_map(c, c->state[k], &c->smap[k], 32, c->fwd.by)) != LBF_OK) return cleanup(st);
    }
  }
  // every grid launch_forward can use must fit the partial sums
  const long long gz = c->fgrid.z;
  for (const KernelInfo* k : {&c->fwd, &c->fwd_tma30, &c->fwd_direct})
    if ((long long)grid_x(c->nx, k->xout) * grid_y(c->ny, k->by) * gz > L.npartials)
      return cleanup(fail(LBF_EINTERNAL, "partials buffer too small"));
  if ((st = setup_split(c, params, L, sms, nearest, kname)) != LBF_OK) return cleanup(st);

  cudaStream_t s = c->stream;
  if (cudaMemsetAsync(c->state[0], 0, 10 * c->N * storage_bytes(c->storage), s) != cudaSuccess ||
      cudaMemsetAsync(c->state[1], 0, 10 * c->N * storage_bytes(c->storage), s) != cudaSuccess ||
      cudaMemsetAsync(c->sums, 0, 64 * sizeof(double), s) != cudaSuccess)
    return cleanup(fail(LBF_ECUDA, "memset failed"));
  if (c->has_mask) {
    if (cudaMemcpyAsync(c->mask_d, params->mask, c->N, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return cleanup(fail(LBF_ECUDA, "mask copy failed"));
  }
  if (c->two) {
    const size_t cb = compute_bytes(c->storage);
    for (int k = 0; k < 2; ++k) {
      if (cudaMemsetAsync(c->phi[k], 0, c->N * cb, s) != cudaSuccess ||
          cudaMemsetAsync(c->F[k], 0, 3 * c->N * cb, s) != cudaSuccess)
        return cleanup(fail(LBF_ECUDA, "memset failed"));
    }
    if (cudaMemsetAsync(c->G, 0, 3 * c->N * cb, s) != cudaSuccess) return cleanup(fail(LBF_ECUDA, "memset failed"));
    if (c->contrast && cudaMemsetAsync(c->gphi, 0, 3 * c->N * cb, s) != cudaSuccess)
      return cleanup(fail(LBF_ECUDA, "memset failed"));
  }
  if (cudaStreamSynchronize(s) != cudaSuccess)
    return cleanup(fail(LBF_ECUDA, std::string("create: ") + cudaGetErrorString(cudaGetLastError())));
  *out = c;
  return LBF_OK;
}

lbf_status lbf_destroy(lbf_ctx* c) {
  if (c != nullptr && c->side != nullptr) {
    cudaStreamSynchronize(c->side);
    cudaEventDestroy(c->ev_fork);
    cudaEventDestroy(c->ev_join);
    cudaStreamDestroy(c->side);
  }
  delete c;
  return LBF_OK;
}

size_t lbf_state_bytes(const lbf_ctx* c) {
  return c ? size_t(c->pops ? c->Q : 10) * c->N * storage_bytes(c->storage) : 0;
}

lbf_status lbf_set_moments(lbf_ctx* c, const void* src, int dt, const void* phi) {
  if (c == nullptr || src == nullptr) return fail(LBF_EINVAL, "NULL argument");
  if (dt != LBF_F64 && dt != LBF_F32) return fail(LBF_EINVAL, "src_dtype must be LBF_F64 or LBF_F32");
  if (c->two && phi == nullptr) return fail(LBF_EINVAL, "two-component state needs phi");
  const bool dev = is_device_pointer(src);
  const size_t eb = dt == LBF_F64 ? 8 : 4;
  const long long N = c->N;
  cudaStream_t s = c->stream;
  if (c->storage == LBF_F16 || c->storage == LBF_BF16) {
    double m[3] = {0, 0, 0};
    // device memory, or pinned host memory read in place by the device
    const void* src_dev = dev ? src : mapped_host_pointer(src);
    if (src_dev != nullptr) {
      LBF_CUDA(cudaMemsetAsync(c->absmax, 0, 3 * sizeof(unsigned), s));
      if (dt == LBF_F64)
        k_absmax<double><<<blocks_for(N, 256), 256, 0, s>>>(static_cast<const double*>(src_dev), N, N, c->absmax);
      else
        k_absmax<float><<<blocks_for(N, 256), 256, 0, s>>>(static_cast<const float*>(src_dev), N, N, c->absmax);
      LBF_CUDA(cudaGetLastError());
      unsigned h[3];
      LBF_CUDA(cudaMemcpyAsync(h, c->absmax, sizeof(h), cudaMemcpyDeviceToHost, s));
      LBF_CUDA(cudaStreamSynchronize(s));
      for (int k = 0; k < 3; ++k) {
        float f;
        std::memcpy(&f, &h[k], sizeof(f));
        m[k] = f;
      }
    } else if (dt == LBF_F64) {
      host_absmax(static_cast<const double*>(src), N, m);
    } else {
      host_absmax(static_cast<const float*>(src), N, m);
    }
    set_scales(c, m);
  }
  void* enc_dst = c->pops ? c->mom : c->state[0];  // populations are built from the moments below
  if (dev) {
    if (dt == LBF_F64) encode_dispatch<double>(c->storage, src, N, 0, N, enc_dst, N, c->sc, s);
    else encode_dispatch<float>(c->storage, src, N, 0, N, enc_dst, N, c->sc, s);
    LBF_CUDA(cudaGetLastError());
  } else if (const void* mapped = mapped_host_pointer(src)) {
    // pinned host memory: the encode pass reads it in place over the host link (one pass)
    if (dt == LBF_F64) encode_dispatch<double>(c->storage, mapped, N, 0, N, enc_dst, N, c->sc, s);
    else encode_dispatch<float>(c->storage, mapped, N, 0, N, enc_dst, N, c->sc, s);
    LBF_CUDA(cudaGetLastError());
  } else if (!c->pops && storage_bytes(c->storage) >= eb) {
    // the second state buffer holds the whole public state: one host copy, then one encode pass
    LBF_CUDA(cudaMemcpyAsync(c->state[1], src, size_t(10) * N * eb, cudaMemcpyHostToDevice, s));
    if (dt == LBF_F64) encode_dispatch<double>(c->storage, c->state[1], N, 0, N, enc_dst, N, c->sc, s);
    else encode_dispatch<float>(c->storage, c->state[1], N, 0, N, enc_dst, N, c->sc, s);
    LBF_CUDA(cudaGetLastError());
  } else {
    const long long chunk = std::max<long long>(1, (long long)(c->lay.staging_bytes / (10 * eb)));
    const unsigned char* h = static_cast<const unsigned char*>(src);
    for (long long s0 = 0; s0 < N; s0 += chunk) {
      const long long cnt = std::min(chunk, N - s0);
      for (int k = 0; k < 10; ++k)
        LBF_CUDA(cudaMemcpyAsync(c->staging + k * cnt * eb, h + (k * N + s0) * eb, cnt * eb, cudaMemcpyHostToDevice, s));
      if (dt == LBF_F64) encode_dispatch<double>(c->storage, c->staging, cnt, s0, cnt, enc_dst, N, c->sc, s);
      else encode_dispatch<float>(c->storage, c->staging, cnt, s0, cnt, enc_dst, N, c->sc, s);
      LBF_CUDA(cudaGetLastError());
    }
  }
  if (c->pops) {
    PopParams pp = pop_params(c, nullptr, c->state[0], false);
    void* args[] = {&pp};
    LBF_CUDA(cudaLaunchKernel(c->popk.init, c->pop_grid, dim3(kPopThreads), args, 0, s));
  }
  LBF_CUDA(cudaMemcpyAsync(c->state[1], c->state[0], lbf_state_bytes(c), cudaMemcpyDeviceToDevice, s));
  c->cur = 0;
  c->pcur = 0;
  if (c->two) {
    const int cd = c->storage == LBF_F64 ? LBF_F64 : LBF_F32;
    const bool pdev = is_device_pointer(phi);
    if (pdev) {
      convert(phi, dt, c->phi[0], cd, N, s);
      LBF_CUDA(cudaGetLastError());
    } else {
      const long long chunk = std::max<long long>(1, (long long)(c->lay.staging_bytes / eb));
      const unsigned char* h = static_cast<const unsigned char*>(phi);
      const size_t cbytes = compute_bytes(c->storage);
      for (long long s0 = 0; s0 < N; s0 += chunk) {
        const long long cnt = std::min(chunk, N - s0);
        LBF_CUDA(cudaMemcpyAsync(c->staging, h + s0 * eb, cnt * eb, cudaMemcpyHostToDevice, s));
        convert(c->staging, dt, static_cast<unsigned char*>(c->phi[0]) + s0 * cbytes, cd, cnt, s);
        LBF_CUDA(cudaGetLastError());
      }
    }
    launch_forces(c, 0);
    LBF_CUDA(cudaGetLastError());
    if (c->contrast) {  // the initial force also holds F^p + F^nu of the loaded state
      const unsigned g = blocks_for(N, 256);
      if (c->storage == LBF_F64)
        k_contrast_init<double, double><<<g, 256, 0, s>>>(static_cast<const double*>(c->state[0]),
                                                          static_cast<const double*>(c->phi[0]),
                                                          static_cast<const double*>(c->gphi), static_cast<double*>(c->F[0]),
                                                          N, c->prm.rho_h - c->prm.rho_l, c->nu_l, c->nu_h - c->nu_l);
      else
        k_contrast_init<float, float><<<g, 256, 0, s>>>(static_cast<const float*>(c->state[0]),
                                                        static_cast<const float*>(c->phi[0]),
                                                        static_cast<const float*>(c->gphi), static_cast<float*>(c->F[0]),
                                                        N, c->prm.rho_h - c->prm.rho_l, c->nu_l, c->nu_h - c->nu_l);
      LBF_CUDA(cudaGetLastError());
    }
  }
  c->sums_valid = false;
  return LBF_OK;
}

lbf_status lbf_step(lbf_ctx* c, int n) {
  if (c == nullptr || n < 0) return fail(LBF_EINVAL, "bad argument");
  for (int i = 0; i < n; ++i) {
    const bool last = i == n - 1;
    if (c->two) {
      launch_advance(c);
      LBF_CUDA(cudaGetLastError());
      launch_forces(c, 1 - c->pcur);
      LBF_CUDA(cudaGetLastError());
    }
    lbf_status st = launch_forward(c, c->state[c->cur], c->state[1 - c->cur], last);
    if (st != LBF_OK) return st;
    c->cur ^= 1;
    if (c->two) c->pcur ^= 1;
  }
  if (n > 0) c->sums_valid = !c->pops;  // the last moment step's kernel wrote them
  return c->unstable_seen ? fail(LBF_EUNSTABLE, "instability flagged by an earlier step") : LBF_OK;
}

lbf_status lbf_step_state(lbf_ctx* c, const void* src, void* dst) {
  if (c == nullptr || src == nullptr || dst == nullptr || src == dst) return fail(LBF_EINVAL, "bad argument");
  if (c->two) return fail(LBF_ENOTSUP, "lbf_step_state is single-component only");
  return launch_forward(c, src, dst, false);
}

lbf_status lbf_moments(lbf_ctx* c, void* dst, int dt, void* phi_dst) {
  if (c == nullptr || dst == nullptr) return fail(LBF_EINVAL, "NULL argument");
  if (dt != LBF_F64 && dt != LBF_F32) return fail(LBF_EINVAL, "dst_dtype must be LBF_F64 or LBF_F32");
  const long long N = c->N;
  const size_t eb = dt == LBF_F64 ? 8 : 4;
  cudaStream_t s = c->stream;
  const void* st = c->state[c->cur];
  if (c->pops) {
    const lbf_status ps = pop_moments(c);
    if (ps != LBF_OK) return ps;
    st = c->mom;
  }
  if (is_device_pointer(dst)) {
    if (dt == LBF_F64) decode_dispatch<double>(c->storage, st, N, 0, N, dst, N, c->sc, s);
    else decode_dispatch<float>(c->storage, st, N, 0, N, dst, N, c->sc, s);
    LBF_CUDA(cudaGetLastError());
  } else if (void* mapped = const_cast<void*>(mapped_host_pointer(dst))) {
    // pinned host memory: the decode pass writes it in place over the host link (one pass)
    if (dt == LBF_F64) decode_dispatch<double>(c->storage, st, N, 0, N, mapped, N, c->sc, s);
    else decode_dispatch<float>(c->storage, st, N, 0, N, mapped, N, c->sc, s);
    LBF_CUDA(cudaGetLastError());
  } else if (!c->pops && storage_bytes(c->storage) >= eb) {
    // decode into the idle state buffer (the next step overwrites it anyway), then one host copy
    void* scratch = c->state[1 - c->cur];
    if (dt == LBF_F64) decode_dispatch<double>(c->storage, st, N, 0, N, scratch, N, c->sc, s);
    else decode_dispatch<float>(c->storage, st, N, 0, N, scratch, N, c->sc, s);
    LBF_CUDA(cudaGetLastError());
    LBF_CUDA(cudaMemcpyAsync(dst, scratch, size_t(10) * N * eb, cudaMemcpyDeviceToHost, s));
    // a step does not write solid sites: the idle buffer must keep their moments
    if (c->has_mask)
      LBF_CUDA(cudaMemcpyAsync(scratch, st, lbf_state_bytes(c), cudaMemcpyDeviceToDevice, s));
  } else {
    const long long chunk = std::max<long long>(1, (long long)(c->lay.staging_bytes / (10 * eb)));
    unsigned char* h = static_cast<unsigned char*>(dst);
    for (long long s0 = 0; s0 < N; s0 += chunk) {
      const long long cnt = std::min(chunk, N - s0);
      if (dt == LBF_F64) decode_dispatch<double>(c->storage, st, N, s0, cnt, c->staging, cnt, c->sc, s);
      else decode_dispatch<float>(c->storage, st, N, s0, cnt, c->staging, cnt, c->sc, s);
      LBF_CUDA(cudaGetLastError());
      for (int k = 0; k < 10; ++k)
        LBF_CUDA(cudaMemcpyAsync(h + (k * N + s0) * eb, c->staging + k * cnt * eb, cnt * eb, cudaMemcpyDeviceToHost, s));
    }
  }
  if (c->two && phi_dst != nullptr) {
    const int cd = c->storage == LBF_F64 ? LBF_F64 : LBF_F32;
    if (is_device_pointer(phi_dst)) {
      convert(c->phi[c->pcur], cd, phi_dst, dt, N, s);
      LBF_CUDA(cudaGetLastError());
    } else {
      const long long chunk = std::max<long long>(1, (long long)(c->lay.staging_bytes / eb));
      const size_t cbytes = compute_bytes(c->storage);
      unsigned char* h = static_cast<unsigned char*>(phi_dst);
      for (long long s0 = 0; s0 < N; s0 += chunk) {
        const long long cnt = std::min(chunk, N - s0);
        convert(static_cast<unsigned char*>(c->phi[c->pcur]) + s0 * cbytes, cd, c->staging, dt, cnt, s);
        LBF_CUDA(cudaGetLastError());
        LBF_CUDA(cudaMemcpyAsync(h + s0 * eb, c->staging, cnt * eb, cudaMemcpyDeviceToHost, s));
      }
    }
  }
  return LBF_OK;
}

#ifdef LBF_DEBUG
lbf_status lbf_debug_wait_probe(lbf_ctx* c, unsigned polls) {
  if (c == nullptr || polls < 1 || polls > kWaitPolls) return fail(LBF_EINVAL, "bad argument");
  k_wait_probe<<<1, 32, 0, c->stream>>>(c->flags, polls);
  LBF_CUDA(cudaGetLastError());
  return LBF_OK;
}
#endif

lbf_status lbf_synchronize(lbf_ctx* c) {
  if (c == nullptr) return fail(LBF_EINVAL, "NULL context");
  // flags[0]: error bits; flags[1], flags[2]: where the first bounded wait gave up (if recorded)
  unsigned f3[4] = {0u, 0u, 0u, 0u};
  LBF_CUDA(cudaMemcpyAsync(f3, c->flags, sizeof(f3), cudaMemcpyDeviceToHost, c->stream));
  LBF_CUDA(cudaStreamSynchronize(c->stream));
  const unsigned f = f3[0];
  const unsigned where[2] = {f3[1], f3[2]};
  // the error bits are reported once: clear them so that the context stays usable
  if (f & 14u) {
    const unsigned keep[4] = {f & 1u, 0u, 0u, 0u};
    LBF_CUDA(cudaMemcpyAsync(c->flags, keep, sizeof(keep), cudaMemcpyHostToDevice, c->stream));
    LBF_CUDA(cudaStreamSynchronize(c->stream));
  }
  if (f & 8u) return fail(LBF_EINTERNAL, "an index check of the LBF_DEBUG build failed");
  if (f & 6u) {
    std::string msg = (f & 4u) ? "a TMA stage was misaligned; the step was abandoned"
                               : "a bounded wait of the step did not complete in time; the step was abandoned";
    if (where[0] & 0x80000000u) {
      static const char* kinds[4] = {"?", "TMA stage", "neighbour row's populations", "freed ring slots"};
      msg += std::string(" (first: ") + kinds[(where[0] >> 24) & 3u] + ", row " + std::to_string((where[0] >> 16) & 0xffu) +
             ", plane " + std::to_string(int(where[0] & 0xffffu)) + " of the chunk, CTA " + std::to_string(where[1]) +
             "; " + std::to_string(f3[3]) + " waits gave up)";
    }
    return fail(LBF_EINTERNAL, msg);
  }
  if (f & 1u) c->unstable_seen = true;
  return c->unstable_seen ? fail(LBF_EUNSTABLE, "non-finite value or |u| > 0.4 in a step") : LBF_OK;
}

lbf_status lbf_reduce(lbf_ctx* c, double* out) {
  if (c == nullptr || out == nullptr) return fail(LBF_EINVAL, "NULL argument");
  if (!c->sums_valid) {
    lbf_status st = reduce_state(c);
    if (st != LBF_OK) return st;
  }
  double h[6];
  LBF_CUDA(cudaMemcpyAsync(h, c->sums, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  lbf_status st = lbf_synchronize(c);
  std::memcpy(out, h, sizeof(h));
  return st;
}

lbf_status lbf_reduce_async(lbf_ctx* c, double* dst) {
  if (c == nullptr || dst == nullptr) return fail(LBF_EINVAL, "NULL argument");
  if (!c->sums_valid) {
    lbf_status st = reduce_state(c);
    if (st != LBF_OK) return st;
  }
  LBF_CUDA(cudaMemcpyAsync(dst, c->sums, 6 * sizeof(double), cudaMemcpyDefault, c->stream));
  return LBF_OK;
}

lbf_status lbf_copy_state(lbf_ctx* c, void* dst) {
  if (c == nullptr || dst == nullptr) return fail(LBF_EINVAL, "NULL argument");
  LBF_CUDA(cudaMemcpyAsync(dst, c->state[c->cur], lbf_state_bytes(c), cudaMemcpyDeviceToDevice, c->stream));
  return LBF_OK;
}

lbf_status lbf_load_state(lbf_ctx* c, const void* src) {
  if (c == nullptr || src == nullptr) return fail(LBF_EINVAL, "NULL argument");
  LBF_CUDA(cudaMemcpyAsync(c->state[c->cur], src, lbf_state_bytes(c), cudaMemcpyDeviceToDevice, c->stream));
  LBF_CUDA(cudaMemcpyAsync(c->state[1 - c->cur], src, lbf_state_bytes(c), cudaMemcpyDeviceToDevice, c->stream));
  c->sums_valid = false;
  return LBF_OK;
}

lbf_status lbf_adjoint_step(lbf_ctx* c, const void* state_t, const void* state_t1, const void* lambda_in,
                            void* lambda_out, double* grad_force) {
  if (c == nullptr || state_t == nullptr || state_t1 == nullptr || lambda_in == nullptr || lambda_out == nullptr ||
      grad_force == nullptr || lambda_in == lambda_out)
    return fail(LBF_EINVAL, "bad argument");
  if (c->two) return fail(LBF_ENOTSUP, "the adjoint is single-component only");
  if (c->pops) return fail(LBF_ENOTSUP, "the adjoint works on the moment representation");
  if (c->Q == LBF_D3Q27H) return fail(LBF_ENOTSUP, "the adjoint is that of the second-order step (D3Q19, D3Q27)");
  if (c->adj.fn == nullptr) return fail(LBF_ENOTSUP, "the adjoint needs LBF_F32 or LBF_F64 storage");
  AdjParams a;
  std::memset(&a, 0, sizeof(a));
  a.state_t = state_t;
  a.state_t1 = state_t1;
  a.lam_in = lambda_in;
  a.lam_out = lambda_out;
  a.grad_force = grad_force;
  a.mask = c->mask_d;
  a.force_field = c->prm.force_field;
  for (int k = 0; k < 3; ++k) a.force[k] = c->prm.force[k];
  a.omega = c->omega;
  a.nx = c->nx;
  a.ny = c->ny;
  a.nz = c->nz;
  a.N = c->N;
  a.sc = c->sc;
  a.zchunk = c->zchunk;
  void* args[] = {&a};
  LBF_CUDA(cudaLaunchKernel(c->adj.fn, c->agrid, dim3(32, c->adj.by + 2, 1), args, c->adj.smem, c->stream));
  return LBF_OK;
}

}  // extern "C"
