// lbf_step_static: one fused step for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs inside another framework's
// allocator or memory pool, callers that must not allocate once their memory plan is fixed, or
// embedders that only ever receive device buffers from elsewhere. lbf_create needs a caller
// workspace; this entry point needs none. It runs one fused stream-collide step from one state
// buffer to another (both owned by the caller) and keeps the per-block reduction partials, the
// block counter and the error flags in a file-scope __device__ array of fixed size, so neither
// the library nor the caller allocates anything.
//
// The array (kStaticScratchBytes) lives on every GPU that loads the library until the process
// exits. All calls share it: two calls that overlap on the GPU (different streams, or host
// threads) race on it; calls on one stream are ordered and safe. The counter and flags it holds
// are cleared at the start of every call with cudaMemsetAsync; after the step the flags word is
// copied to the caller's flags_device (when given) with a device-to-device cudaMemcpyAsync, so a
// caller without a context still learns whether the step was abandoned or went unstable.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/lbf.h"
#include "dispatch.cuh"

using namespace lbf;

namespace {

constexpr int kStaticMaxBlocks = 16384;  // CTAs of one step: gx * gy * z-chunks
constexpr size_t kStaticHeader = 256;    // sums are written to the caller; counter, flags here
constexpr size_t kStaticScratchBytes = kStaticHeader + size_t(kStaticMaxBlocks) * 8 * sizeof(double);

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

thread_local std::string g_static_error;

lbf_status static_fail(lbf_status s, const std::string& m) {
  g_static_error = m;
  return s;
}

// once per device, with that device current: the device address of the static array. Host code
// must not use the array's name as an address (it is a host-side stand-in).
lbf_status scratch_for_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return static_fail(LBF_ECUDA, "cudaGetDevice failed or device index out of range");
  std::lock_guard<std::mutex> lock(g_mutex);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return static_fail(LBF_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return LBF_OK;
}

}  // namespace

namespace {

PFN_cuTensorMapEncodeTiled_v12000 static_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  std::lock_guard<std::mutex> lock(g_mutex);
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

}  // namespace

void lbf_internal_set_last_error(const char* msg);

extern "C" lbf_status lbf_step_static(const lbf_params* params, const void* src, void* dst,
                                      const uint8_t* mask_device, double* sums_device, unsigned* flags_device) {
  auto fail = [](lbf_status s, const std::string& m) {
    lbf_internal_set_last_error(m.c_str());
    return s;
  };
  lbf_status st = lbf_validate(params);
  if (st != LBF_OK) return st;
  if (params->two_component) return fail(LBF_ENOTSUP, "lbf_step_static is single-component only");
  if (params->populations) return fail(LBF_ENOTSUP, "lbf_step_static works on the moment representation");
  if (params->storage != LBF_F32 && params->storage != LBF_F64)
    return fail(LBF_ENOTSUP, "lbf_step_static needs LBF_F32 or LBF_F64 storage (16-bit scales live in a context)");
  if (src == nullptr || dst == nullptr || src == dst) return fail(LBF_EINVAL, "src and dst must be distinct device buffers");

  const int nx = params->nx, ny = params->ny, nz = params->nz;
  const long long N = (long long)nx * ny * nz;
  const size_t es = params->storage == LBF_F64 ? 8 : 4;
  PFN_cuTensorMapEncodeTiled_v12000 enc = static_encoder();
  // TMA needs 16-byte row strides and a 16-byte aligned base; other buffers (e.g. a view into a
  // larger tensor) take the kernel that loads every site directly
  const bool tma = enc != nullptr && (size_t(nx) * es) % 16 == 0 && reinterpret_cast<uintptr_t>(src) % 16 == 0 &&
                   std::getenv("LBF_NO_TMA") == nullptr;
  const KernelInfo k = forward_kernel_for(params->lattice, params->storage, mask_device != nullptr, false,
                                          params->force_field != nullptr, tma, false);
  if (k.fn == nullptr) return fail(LBF_ENOTSUP, "no kernel for this combination");

  // grid: 30 x by output columns per CTA, z-chunks of about 32 planes, at most kStaticMaxBlocks CTAs
  const long long tiles = (long long)((nx + 29) / 30) * ((ny + k.by - 1) / k.by);
  if (tiles > kStaticMaxBlocks)
    return fail(LBF_EINVAL, "lattice too wide for lbf_step_static: ceil(nx/30)*ceil(ny/" + std::to_string(k.by) +
                                ") = " + std::to_string(tiles) + " exceeds " + std::to_string(kStaticMaxBlocks) +
                                " (" + std::to_string(k.by) + " = output rows per CTA of this kernel)");
  int zc = std::min(nz, 32);
  const long long max_chunks = kStaticMaxBlocks / tiles;
  if ((nz + zc - 1) / zc > max_chunks) zc = int((nz + max_chunks - 1) / max_chunks);
  const dim3 grid((nx + 29) / 30, (ny + k.by - 1) / k.by, (nz + zc - 1) / zc);

  void* scratch = nullptr;
  if ((st = scratch_for_current_device(&scratch)) != LBF_OK) return fail(st, g_static_error);
  unsigned* counter = static_cast<unsigned*>(scratch);
  unsigned* flags = counter + 1;
  double* partials = reinterpret_cast<double*>(static_cast<unsigned char*>(scratch) + kStaticHeader);
  cudaStream_t stream = static_cast<cudaStream_t>(params->stream);
  cudaError_t e = cudaMemsetAsync(scratch, 0, kStaticHeader, stream);  // counter and flags start at zero
  if (e != cudaSuccess) return fail(LBF_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));

  FwdParams a;
  std::memset(&a, 0, sizeof(a));
  a.src = src;
  a.dst = dst;
  a.mask = mask_device;
  a.force_field = params->force_field;
  for (int i = 0; i < 3; ++i) a.force[i] = params->force[i];
  a.omega = 1.0 / params->tau;
  a.nx = nx;
  a.ny = ny;
  a.nz = nz;
  a.N = N;
  for (int g = 0; g < 3; ++g) a.sc.enc[g] = a.sc.dec[g] = 1.0f;
  a.partials = sums_device ? partials : nullptr;
  a.sums = sums_device;
  a.counter = counter;
  a.flags = flags;
  a.zchunk = zc;
  a.umax2 = 0.16f;
  set_fp32_copies(a);

  CUtensorMap tm;
  std::memset(&tm, 0, sizeof(tm));
  if (tma) {
    const cuuint64_t dims[4] = {cuuint64_t(nx), cuuint64_t(ny), cuuint64_t(nz), 10};
    const cuuint64_t strides[3] = {es * nx, es * nx * ny, es * cuuint64_t(N)};
    const cuuint32_t box[4] = {cuuint32_t(k.box_x), cuuint32_t(k.by + 2), 1, 10};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = enc(&tm, params->storage == LBF_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                           4, const_cast<void*>(src), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(LBF_ECUDA, "cuTensorMapEncodeTiled failed with code " + std::to_string(int(r)));
  }
  if ((e = cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(k.smem))) != cudaSuccess ||
      (e = cudaFuncSetAttribute(k.fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100)) != cudaSuccess)
    return fail(LBF_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
  void* args[] = {&a, &tm};
  if ((e = cudaLaunchKernel(k.fn, grid, dim3(32, k.by + 2, 1), args, k.smem, stream)) != cudaSuccess)
    return fail(LBF_ECUDA, std::string("cudaLaunchKernel: ") + cudaGetErrorString(e));
  if (flags_device != nullptr &&
      (e = cudaMemcpyAsync(flags_device, flags, sizeof(unsigned), cudaMemcpyDeviceToDevice, stream)) != cudaSuccess)
    return fail(LBF_ECUDA, std::string("cudaMemcpyAsync (flags): ") + cudaGetErrorString(e));
  return LBF_OK;
}
