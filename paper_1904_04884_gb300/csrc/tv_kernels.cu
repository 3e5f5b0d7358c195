// Fused-lasso prox and FISTA update kernels (Section 2: TV prox by
// Beck-Teboulle gradient projection, soft threshold, accelerated update).
//
// TV dual step, per voxel (isotropic TV, forward differences D with Neumann
// boundary, complex values treated as R^2):
//     u  = v - mu * D^H p
//     p' = Pi( p + step * D u ),   step = 1 / (4 dims mu)
// where (D_x^H p)_i = p_{i-1} [i >= 1] - p_i [i <= n-2] (same along y and z)
// and Pi scales the voxel's (p_x, p_y, p_z) in C^3 onto the unit ball.
//
// k_tv_step marches a 32x8 x-y tile through a chunk of planes (2.5D blocking).
// Each plane of v, p_x, p_y, p_z arrives in shared memory as one TMA box
// (x from i0-2, y from j0-1: the stencil's halo, with the x start kept on a
// 16-byte boundary; out-of-range boxes are zero filled) into a 4-stage ring
// completed by mbarriers, so two planes are in flight while one is computed.
// u is formed for plane k+1 over the tile plus its +x/+y halo, then p' of
// plane k is written with plain coalesced stores. Every wait is bounded: on
// timeout the CTA sets the error flag, drains its copies in flight and exits.
//
// The finalize kernel forms u = v - mu D^H p, soft-thresholds it, and (in
// FISTA mode) writes x_k and y_{k+1} = x_k + beta (x_k - x_{k-1}) and reduces
// the gradient-restart inner product Re<y_k - x_k, x_k - x_{k-1}> in FP64.
// The last block of the grid (ticket counter) updates t, beta and the restart
// flag on the device, so no scalar crosses to the host.
#include <cuda_runtime.h>

#include "rihv_internal.cuh"

namespace rihv {
namespace {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

constexpr int TX = kTvTx;
constexpr int TY = kTvTy;
constexpr int RX = TX + 1;        // region of u: tile plus +x / +y halo
constexpr int RY = TY + 1;
constexpr int BW = kTvBoxW;       // TMA box: complex x in [i0-2, i0+TX+2)
constexpr int BH = kTvBoxH;       //          y in [j0-1, j0+TY]
constexpr int NSTAGE = kTvStages;
constexpr int SLOT = kTvSlotBytes;
constexpr int kWaitLimit = 1 << 22;   // bounded mbarrier polls before giving up

// ---- PTX helpers (TMA + mbarrier) -----------------------------------------
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: true if the phase completed, false after kWaitLimit polls.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
  for (int it = 0; it < kWaitLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void tma_load_3d(unsigned dst, const CUtensorMap* tm, int x, int y, int z,
                                            unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<unsigned long long>(tm)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// Shared memory: NSTAGE stages x 4 slots (v, p_x, p_y, p_z) of one box each,
// then the two u planes, then the mbarriers.
struct TvLayout {
  static constexpr int kStageBytes = 4 * SLOT;
  static constexpr int kUBytes = 2 * RY * RX * 8;
  static constexpr int kBarOffset = NSTAGE * kStageBytes + kUBytes;
  static constexpr int kBytes = kBarOffset + NSTAGE * 8;
};

template <bool FIRST>
__global__ void __launch_bounds__(kTvThreads) k_tv_step(const __grid_constant__ TvArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  float2(*U)[RY][RX] = reinterpret_cast<float2(*)[RY][RX]>(smem + NSTAGE * TvLayout::kStageBytes);
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(smem + TvLayout::kBarOffset);

  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int zc0 = blockIdx.z * a.zchunk;
  const int zc1 = min(a.nz, zc0 + a.zchunk);
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int gi = i0 + tx, gj = j0 + ty;
  const int base = zc0 - 1;                // plane held by stage 0, use 0
  const int qlast = min(zc1, a.nz - 1);    // last plane this CTA needs
  const int nslots = FIRST ? 1 : (a.dims == 3 ? 4 : 3);

  auto slot = [&](int q, int arr) -> float2(*)[BW] {
    const int s = (q - base) & (NSTAGE - 1);
    return reinterpret_cast<float2(*)[BW]>(smem + s * TvLayout::kStageBytes + arr * SLOT);
  };
  auto bar_of = [&](int q) { return smem_addr(&bars[(q - base) & (NSTAGE - 1)]); };
  auto parity_of = [&](int q) { return static_cast<unsigned>(((q - base) / NSTAGE) & 1); };
  auto issue = [&](int q) {      // thread 0 only
    const unsigned bar = bar_of(q);
    mbar_expect_tx(bar, static_cast<unsigned>(nslots * BW * BH * 8));
    const int x = 2 * (i0 - 2), y = j0 - 1;
    tma_load_3d(smem_addr(slot(q, 0)), &a.tm_v, x, y, q, bar);
    if (!FIRST) {
      tma_load_3d(smem_addr(slot(q, 1)), &a.tm_p[0], x, y, q, bar);
      tma_load_3d(smem_addr(slot(q, 2)), &a.tm_p[1], x, y, q, bar);
      if (a.dims == 3) tma_load_3d(smem_addr(slot(q, 3)), &a.tm_p[2], x, y, q, bar);
    }
  };

  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) mbar_init(smem_addr(&bars[s]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  int issued = base - 1;
  if (tid == 0) {
    for (int q = base; q < base + NSTAGE && q <= qlast; ++q) issue(q);
  }
  issued = min(base + NSTAGE - 1, qlast);
  int waited = base - 1;

  // u(k) over the region from stage(k) (p, v) and stage(k-1) (p_z).
  auto form_u = [&](int k) {
    float2(*vs)[BW] = slot(k, 0);
    float2(*px)[BW] = slot(k, 1);
    float2(*py)[BW] = slot(k, 2);
    float2(*pz)[BW] = slot(k, 3);
    float2(*pzm)[BW] = slot(k - 1, 3);
    float2(*u)[RX] = U[k & 1];
    for (int e = tid; e < RY * RX; e += kTvThreads) {
      const int ry = e / RX, rx = e - ry * RX;
      const int gx = i0 + rx, gy = j0 + ry;
      const int by = ry + 1, bx = rx + 2;
      float2 uu = vs[by][bx];
      if (!FIRST) {
        float2 dh = make_float2(0.f, 0.f);
        if (gx >= 1) dh = cadd(dh, px[by][bx - 1]);
        if (gx <= a.nx - 2) dh = csub(dh, px[by][bx]);
        if (gy >= 1) dh = cadd(dh, py[by - 1][bx]);
        if (gy <= a.ny - 2) dh = csub(dh, py[by][bx]);
        if (a.dims == 3) {
          if (k >= 1) dh = cadd(dh, pzm[by][bx]);
          if (k <= a.nz - 2) dh = csub(dh, pz[by][bx]);
        }
        uu = make_float2(uu.x - a.mu * dh.x, uu.y - a.mu * dh.y);
      }
      u[ry][rx] = uu;
    }
  };
  auto wait_plane = [&](int q) -> bool {
    const bool ok = mbar_wait(bar_of(q), parity_of(q));
    return __syncthreads_and(ok) != 0;
  };
  auto abort_drain = [&]() {
    // Record the failure and wait (bounded) for this CTA's copies in flight
    // before its shared memory is released.
    if (tid == 0) {
      atomicExch(a.err, 1);
      for (int q = waited + 1; q <= issued; ++q) mbar_wait(bar_of(q), parity_of(q));
    }
    __syncthreads();
  };

  // prologue: planes base (p_z only) and zc0
  if (!wait_plane(base)) { abort_drain(); return; }
  if (!wait_plane(zc0)) { waited = base; abort_drain(); return; }
  waited = zc0;
  form_u(zc0);
  __syncthreads();

  for (int k = zc0; k < zc1; ++k) {
    // stage of plane k-1 is free: refill it with plane k+3
    if (k + 3 <= qlast) {
      if (tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(k + 3);
      }
      issued = k + 3;
    }
    const bool has_next = (k + 1 < a.nz);
    if (has_next) {
      if (!wait_plane(k + 1)) { abort_drain(); return; }
      waited = k + 1;
      form_u(k + 1);
    }
    __syncthreads();
    if (gi < a.nx && gj < a.ny) {
      float2(*u)[RX] = U[k & 1];
      float2(*un)[RX] = U[(k + 1) & 1];
      const float2 u0 = u[ty][tx];
      float2 gx = make_float2(0.f, 0.f), gy = gx, gz = gx;
      if (gi <= a.nx - 2) gx = csub(u[ty][tx + 1], u0);
      if (gj <= a.ny - 2) gy = csub(u[ty + 1][tx], u0);
      if (a.dims == 3 && k <= a.nz - 2) gz = csub(un[ty][tx], u0);
      float2 qx, qy, qz;
      if (FIRST) {
        qx = make_float2(a.step * gx.x, a.step * gx.y);
        qy = make_float2(a.step * gy.x, a.step * gy.y);
        qz = make_float2(a.step * gz.x, a.step * gz.y);
      } else {
        const int by = ty + 1, bx = tx + 2;
        const float2 ox = slot(k, 1)[by][bx];
        const float2 oy = slot(k, 2)[by][bx];
        const float2 oz = (a.dims == 3) ? slot(k, 3)[by][bx] : make_float2(0.f, 0.f);
        qx = make_float2(ox.x + a.step * gx.x, ox.y + a.step * gx.y);
        qy = make_float2(oy.x + a.step * gy.x, oy.y + a.step * gy.y);
        qz = make_float2(oz.x + a.step * gz.x, oz.y + a.step * gz.y);
      }
      const float n2 = qx.x * qx.x + qx.y * qx.y + qy.x * qy.x + qy.y * qy.y + qz.x * qz.x + qz.y * qz.y;
      if (n2 > 1.f) {
        const float sc = rsqrtf(n2);
        qx.x *= sc; qx.y *= sc; qy.x *= sc; qy.y *= sc; qz.x *= sc; qz.y *= sc;
      }
      const size_t gidx = (static_cast<size_t>(k) * a.ny + gj) * a.nx + gi;
      a.pout[0][gidx] = qx;
      a.pout[1][gidx] = qy;
      if (a.dims == 3) a.pout[2][gidx] = qz;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (wid == 0) {
    r = (lane < static_cast<int>(blockDim.x >> 5)) ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  }
  __syncthreads();
  return r;
}

// Writes this block's partial (slot `which`) and returns true in every thread
// of the last block to arrive, which then owns the final sum.
__device__ __forceinline__ bool publish_partial(double bs, RedWork w, int which, int ticket) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    w.partials[which * kRedBlocks + blockIdx.x] = bs;
    __threadfence();
    last = atomicAdd(&w.tickets[ticket], 1u) == gridDim.x - 1;
  }
  __syncthreads();
  return last;
}

__device__ __forceinline__ double final_sum(RedWork w, int which) {
  __threadfence();
  double v = 0.0;
  for (int b = threadIdx.x; b < static_cast<int>(gridDim.x); b += blockDim.x)
    v += static_cast<volatile double*>(w.partials)[which * kRedBlocks + b];
  return block_sum(v);
}

// u = v - mu D^H p at voxel (i, j, k), straight from global memory.
__device__ __forceinline__ float2 form_u(const FinArgs& a, size_t idx, int i, int j, int k) {
  float2 u = a.v[idx];
  if (a.p[0]) {
    const size_t sy = a.nx, sz = static_cast<size_t>(a.nx) * a.ny;
    float2 dh = make_float2(0.f, 0.f);
    if (i >= 1) dh = cadd(dh, a.p[0][idx - 1]);
    if (i <= a.nx - 2) dh = csub(dh, a.p[0][idx]);
    if (j >= 1) dh = cadd(dh, a.p[1][idx - sy]);
    if (j <= a.ny - 2) dh = csub(dh, a.p[1][idx]);
    if (a.dims == 3) {
      if (k >= 1) dh = cadd(dh, a.p[2][idx - sz]);
      if (k <= a.nz - 2) dh = csub(dh, a.p[2][idx]);
    }
    u = make_float2(u.x - a.mu * dh.x, u.y - a.mu * dh.y);
  }
  return u;
}

__device__ __forceinline__ float2 soft(float2 u, float kappa) {
  const float mag = sqrtf(u.x * u.x + u.y * u.y);
  const float s = (mag > kappa) ? (1.f - kappa / mag) : 0.f;
  return make_float2(u.x * s, u.y * s);
}

template <int MODE>
__global__ void __launch_bounds__(kRedThreads) k_finalize(const __grid_constant__ FinArgs a) {
  const size_t nvox = static_cast<size_t>(a.nx) * a.ny * a.nz;
  const float beta = (MODE == FIN_FISTA) ? static_cast<float>(a.sc->beta) : 0.f;
  float local = 0.f;
  double dsum = 0.0;
  int cnt = 0;
  for (size_t idx = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; idx < nvox;
       idx += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int i = static_cast<int>(idx % a.nx);
    const size_t r = idx / a.nx;
    const int j = static_cast<int>(r % a.ny);
    const int k = static_cast<int>(r / a.ny);
    const float2 x = soft(form_u(a, idx, i, j, k), a.kappa);
    if (MODE == FIN_FISTA) {
      const float2 xp = a.x_prev[idx];
      const float2 yk = a.y[idx];
      const float2 dx = csub(x, xp);
      local += (yk.x - x.x) * dx.x + (yk.y - x.y) * dx.y;
      if (++cnt == 8) { dsum += local; local = 0.f; cnt = 0; }
      a.y_out[idx] = make_float2(x.x + beta * dx.x, x.y + beta * dx.y);
    }
    a.x_out[idx] = x;
  }
  if (MODE != FIN_FISTA) return;
  dsum += local;
  const double bs = block_sum(dsum);
  if (!publish_partial(bs, a.w, 0, 1)) return;
  const double dot = final_sum(a.w, 0);
  if (threadIdx.x == 0) {
    DevScalars* sc = a.sc;
    sc->restart_dot = dot;
    if (!isfinite(dot)) sc->nonfinite = 1;
    double t = sc->t;
    int restart = 0;
    if (sc->accelerate) {
      double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
      if (sc->restart && dot > 0.0) {
        tn = 1.0;
        restart = 1;
      }
      t = tn;
      const double t2 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
      sc->beta = (t - 1.0) / t2;
    } else {
      t = 1.0;
      sc->beta = 0.0;
    }
    sc->t = t;
    sc->restart_flag = restart;
    a.w.tickets[1] = 0;
  }
}

__global__ void k_restart_fixup(const float2* x, float2* y, size_t nvox, const DevScalars* sc) {
  if (!sc->restart_flag) return;
  for (size_t idx = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; idx < nvox;
       idx += static_cast<size_t>(gridDim.x) * blockDim.x)
    y[idx] = x[idx];
}

__global__ void __launch_bounds__(kRedThreads) k_objective(const float2* x, int nx, int ny, int nz,
                                                           int dims, double lam_l1, double lam_tv,
                                                           DevScalars* sc, RedWork w, double* f_out) {
  const size_t nvox = static_cast<size_t>(nx) * ny * nz;
  const size_t sy = nx, sz = static_cast<size_t>(nx) * ny;
  float l1 = 0.f, tv = 0.f;
  double dl1 = 0.0, dtv = 0.0;
  int cnt = 0;
  for (size_t idx = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; idx < nvox;
       idx += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int i = static_cast<int>(idx % nx);
    const size_t r = idx / nx;
    const int j = static_cast<int>(r % ny);
    const int k = static_cast<int>(r / ny);
    const float2 c = x[idx];
    l1 += sqrtf(c.x * c.x + c.y * c.y);
    float g2 = 0.f;
    if (i <= nx - 2) { const float2 d = csub(x[idx + 1], c); g2 += d.x * d.x + d.y * d.y; }
    if (j <= ny - 2) { const float2 d = csub(x[idx + sy], c); g2 += d.x * d.x + d.y * d.y; }
    if (dims == 3 && k <= nz - 2) { const float2 d = csub(x[idx + sz], c); g2 += d.x * d.x + d.y * d.y; }
    tv += sqrtf(g2);
    if (++cnt == 8) { dl1 += l1; dtv += tv; l1 = 0.f; tv = 0.f; cnt = 0; }
  }
  dl1 += l1;
  dtv += tv;
  const double b1 = block_sum(dl1);
  const double b2 = block_sum(dtv);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    w.partials[1 * kRedBlocks + blockIdx.x] = b1;
    w.partials[2 * kRedBlocks + blockIdx.x] = b2;
    __threadfence();
    last = atomicAdd(&w.tickets[2], 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  const double s1 = final_sum(w, 1);
  const double s2 = final_sum(w, 2);
  if (threadIdx.x == 0) {
    sc->l1 = s1;
    sc->tv = s2;
    const double f = sc->rnorm2 + lam_l1 * s1 + lam_tv * s2;
    if (!isfinite(f)) sc->nonfinite = 1;
    *f_out = f;
    w.tickets[2] = 0;
  }
}

__global__ void k_init_scalars(DevScalars* sc, int accelerate, int restart) {
  sc->t = 1.0;
  sc->beta = 0.0;  // (t_1 - 1) / t_2 with t_1 = 1
  sc->restart_dot = 0.0;
  sc->rnorm2 = 0.0;
  sc->l1 = 0.0;
  sc->tv = 0.0;
  sc->restart_flag = 0;
  sc->nonfinite = 0;
  sc->accelerate = accelerate;
  sc->restart = restart;
}

int stream_grid(size_t nvox) {
  size_t b = (nvox + kRedThreads - 1) / kRedThreads;
  return static_cast<int>(b < static_cast<size_t>(kRedBlocks) ? b : kRedBlocks);
}

}  // namespace

cudaError_t launch_tv_step(bool first, const TvArgs& a, cudaStream_t s) {
  dim3 grid((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY, (a.nz + a.zchunk - 1) / a.zchunk);
  auto kern = first ? k_tv_step<true> : k_tv_step<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       TvLayout::kBytes);
  if (e != cudaSuccess) return e;
  kern<<<grid, kTvThreads, TvLayout::kBytes, s>>>(a);
  return cudaGetLastError();
}

// 3D tensor map over a complex64 volume viewed as float32 [nz][ny][2 nx], box
// of kTvBoxH rows x 2 kTvBoxW floats x 1 plane, zero fill out of bounds.
cudaError_t make_volume_tmap(CUtensorMap* tm, const void* base, int nx, int ny, int nz) {
  using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static EncodeFn encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = reinterpret_cast<EncodeFn>(fn);
  }
  const cuuint64_t dims[3] = {static_cast<cuuint64_t>(2 * nx), static_cast<cuuint64_t>(ny),
                              static_cast<cuuint64_t>(nz)};
  const cuuint64_t strides[2] = {static_cast<cuuint64_t>(8) * nx,
                                 static_cast<cuuint64_t>(8) * nx * ny};
  const cuuint32_t box[3] = {2 * kTvBoxW, kTvBoxH, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = encode(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims,
                      strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_finalize(int mode, const FinArgs& a, cudaStream_t s) {
  const size_t nvox = static_cast<size_t>(a.nx) * a.ny * a.nz;
  const int grid = stream_grid(nvox);
  if (mode == FIN_FISTA)
    k_finalize<FIN_FISTA><<<grid, kRedThreads, 0, s>>>(a);
  else
    k_finalize<FIN_PROX><<<grid, kRedThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_restart_fixup(const float2* x, float2* y, size_t nvox, const DevScalars* sc,
                                 cudaStream_t s) {
  k_restart_fixup<<<stream_grid(nvox), kRedThreads, 0, s>>>(x, y, nvox, sc);
  return cudaGetLastError();
}

cudaError_t launch_objective(const float2* x, int nx, int ny, int nz, int dims, double lam_l1,
                             double lam_tv, DevScalars* sc, RedWork w, double* f_out,
                             cudaStream_t s) {
  const size_t nvox = static_cast<size_t>(nx) * ny * nz;
  k_objective<<<stream_grid(nvox), kRedThreads, 0, s>>>(x, nx, ny, nz, dims, lam_l1, lam_tv, sc, w,
                                                         f_out);
  return cudaGetLastError();
}

cudaError_t launch_init_scalars(DevScalars* sc, int accelerate, int restart, cudaStream_t s) {
  k_init_scalars<<<1, 1, 0, s>>>(sc, accelerate, restart);
  return cudaGetLastError();
}

}  // namespace rihv
