// rihv_prox_fused_lasso_noalloc: the fused-lasso prox for callers that must
// not allocate device memory.
//
// Some callers cannot call cudaMalloc: hosts whose device memory is a fixed
// arena handed out by another framework (the library may not take memory
// behind its back), and services that lock their allocator after start-up so
// that no request can fail, or stall on a device-wide synchronisation, for
// lack of memory. For them this file keeps the prox's scratch (the two
// ping-pong sets of the TV dual variable and an error flag) in one statically
// sized device array that the CUDA driver reserves when the library's module
// is loaded on a device, and that every call reuses. The caller still passes
// the input and output volumes.
//
// Limit: nx * ny * nz <= kNoAllocMaxVoxels (1,048,576 voxels, e.g.
// 128 x 128 x 64); the scratch is 6 x 8 MiB + 256 B and stays reserved on
// every GPU that loads the library until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "rihv_internal.cuh"

namespace {

constexpr size_t kNoAllocMaxVoxels = static_cast<size_t>(1) << 20;
constexpr size_t kDualBytes = 6 * kNoAllocMaxVoxels * sizeof(float2);
constexpr size_t kScratchBytes = kDualBytes + 256;   // + error flag

// The scratch itself. In host code this name is only a stand-in for the
// device array: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};
// The status code carries the outcome; the reason goes to rihv_last_error(NULL).
rihv_status fail(rihv_status st, const char* why) {
  rihv::set_global_error(why);
  return st;
}

// Device address of the scratch on the current device (looked up once per
// device, with that device current).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

// A TV kernel whose bounded wait gave up left its flag in the scratch. The
// call has already returned, so the output itself carries the failure: every
// voxel becomes NaN, which no finite prox result contains. With the flag
// clear (the normal case) each thread reads one word and exits.
__global__ void k_poison_on_timeout(const int* err, float2* x, size_t nvox) {
  if (*err == 0) return;
  const float nan = __int_as_float(0x7fc00000);
  for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < nvox;
       i += static_cast<size_t>(gridDim.x) * blockDim.x)
    x[i] = make_float2(nan, nan);
}

}  // namespace

extern "C" rihv_status rihv_prox_fused_lasso_noalloc(const void* v, void* x_out, int nx, int ny,
                                                     int nz, int tv_dims, float t_l1, float t_tv,
                                                     int inner_iters, void* stream) {
  using namespace rihv;
  if (nx < 2 || ny < 1 || nz < 1 || (nx % 2) != 0)
    return fail(RIHV_ERR_INVALID_ARG, "nx must be even and >= 2, ny and nz >= 1");
  const size_t nvox = static_cast<size_t>(nx) * ny * nz;
  if (nvox > kNoAllocMaxVoxels)
    return fail(RIHV_ERR_UNSUPPORTED_SIZE, "volume exceeds the no-allocation limit");
  if (tv_dims != 2 && tv_dims != 3) return fail(RIHV_ERR_INVALID_ARG, "tv_dims must be 2 or 3");
  if (!(t_l1 >= 0.f) || !(t_tv >= 0.f) || !std::isfinite(t_l1) || !std::isfinite(t_tv) ||
      inner_iters < 0)
    return fail(RIHV_ERR_INVALID_ARG, "t_l1, t_tv must be finite and >= 0, inner_iters >= 0");
  if (!v || !x_out || v == x_out) return fail(RIHV_ERR_INVALID_ARG, "v, x_out: distinct, non-NULL");
  if ((reinterpret_cast<uintptr_t>(v) & 15u) || (reinterpret_cast<uintptr_t>(x_out) & 15u))
    return fail(RIHV_ERR_INVALID_ARG, "v and x_out must be 16-byte aligned");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(RIHV_ERR_CUDA, "cudaGetDevice failed");
  // The scratch looked up below is the current device's, so the volumes and
  // the stream must be on that device too (memory of another GPU would be
  // read through peer access, or fault).
  for (const void* p : {v, static_cast<const void*>(x_out)}) {
    const int where = pointer_device(p);
    if (where == kNotDevicePtr) return fail(RIHV_ERR_INVALID_ARG, "v and x_out must be device memory");
    if (where != kManagedPtr && where != dev)
      return fail(RIHV_ERR_INVALID_ARG, "v or x_out lives on another device than the current one");
  }
  const int sd = stream_device(stream);
  if (sd != kLegacyStream && sd != dev)
    return fail(RIHV_ERR_INVALID_ARG, "the stream belongs to another device than the current one");

  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess)
    return fail(RIHV_ERR_CUDA, "cudaGetSymbolAddress of the no-allocation scratch failed");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float2* duals = static_cast<float2*>(base);
  int* err = reinterpret_cast<int*>(static_cast<unsigned char*>(base) + kDualBytes);
  float2* pa[3];
  float2* pb[3];
  for (int c = 0; c < 3; ++c) {
    pa[c] = duals + static_cast<size_t>(c) * nvox;
    pb[c] = duals + static_cast<size_t>(3 + c) * nvox;
  }
  if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess)
    return fail(RIHV_ERR_CUDA, "clearing the error flag failed");

  const bool tv = (t_tv > 0.f && inner_iters > 0);
  float2* const* pfinal = nullptr;
  if (tv) {
    TvArgs a{};
    if (make_volume_tmap(&a.tm_v, v, nx, ny, nz, kTvBoxH1, kTvBoxW) != cudaSuccess)
      return fail(RIHV_ERR_CUDA, "tensor map encoding failed");
    CUtensorMap tma[3], tmb[3];
    for (int c = 0; c < 3; ++c)
      if (make_volume_tmap(&tma[c], pa[c], nx, ny, nz, kTvBoxH1, kTvBoxW) != cudaSuccess ||
          make_volume_tmap(&tmb[c], pb[c], nx, ny, nz, kTvBoxH1, kTvBoxW) != cudaSuccess)
        return fail(RIHV_ERR_CUDA, "tensor map encoding failed");
    a.err = err;
    a.nx = nx;
    a.ny = ny;
    a.nz = nz;
    a.dims = tv_dims;
    a.zchunk = 32;
    a.mu = t_tv;
    a.step = 1.f / (4.f * tv_dims * t_tv);
    float2** src = pb;
    float2** dst = pa;
    const CUtensorMap* tsrc = tmb;
    const CUtensorMap* tdst = tma;
    for (int it = 0; it < inner_iters; ++it) {
      for (int c = 0; c < 3; ++c) {
        a.tm_p[c] = tsrc[c];
        a.pout[c] = dst[c];
      }
      if (launch_tv_step(it == 0, 1, a, s) != cudaSuccess)
        return fail(RIHV_ERR_CUDA, "TV step launch failed");
      float2** t = src;
      src = dst;
      dst = t;
      const CUtensorMap* tt = tsrc;
      tsrc = tdst;
      tdst = tt;
    }
    pfinal = src;
  }
  FinArgs f{};
  f.v = static_cast<const float2*>(v);
  for (int c = 0; c < 3; ++c) f.p[c] = tv ? pfinal[c] : nullptr;
  f.x_out = static_cast<float2*>(x_out);
  f.nx = nx;
  f.ny = ny;
  f.nz = nz;
  f.dims = tv_dims;
  f.mu = tv ? t_tv : 0.f;
  f.kappa = t_l1;
  if (launch_finalize(FIN_PROX, f, s) != cudaSuccess)
    return fail(RIHV_ERR_CUDA, "finalize launch failed");
  if (tv) {
    k_poison_on_timeout<<<2 * 152, 256, 0, s>>>(err, static_cast<float2*>(x_out), nvox);
    if (cudaGetLastError() != cudaSuccess) return fail(RIHV_ERR_CUDA, "launch failed");
  }
  return RIHV_OK;
}
