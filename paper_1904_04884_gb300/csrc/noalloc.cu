// rihv_prox_fused_lasso_noalloc: the fused-lasso prox for callers that must
// not allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs while a CUDA graph is
// being captured (allocation is not allowed inside a capture), hosts whose
// memory is a fixed arena handed out by another framework, and services that
// lock their allocator after start-up so that no request can fail on memory.
// For them this file keeps the prox's scratch (the two ping-pong sets of the
// TV dual variable) in one statically sized device array that the CUDA driver
// reserves when the library's module is loaded on a device, and that every
// call reuses. The caller still passes the input and output volumes.
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
rihv_status fail(rihv_status st, const char* why) {
  (void)why;   // the status code carries the outcome; see include/rihv.h
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

bool is_device(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
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
  if (!is_device(v) || !is_device(x_out))
    return fail(RIHV_ERR_INVALID_ARG, "v and x_out must be device memory");

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
  return RIHV_OK;
}
