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
// k_tv_step marches a 32x8 x-y tile through a chunk of planes (2.5D blocking):
// plane k+1's p and v are staged in shared memory together with the halo the
// stencil needs (x-1 for p_x, y-1 for p_y, and plane k for p_z), u is formed
// for plane k+1 over the tile plus its +x/+y halo, and p' of plane k is
// written. Each p and v value is read from HBM about once per step.
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
constexpr int RX = TX + 1;   // region of u: tile plus +x / +y halo
constexpr int RY = TY + 1;

struct TvSmem {
  float2 px[2][RY][TX + 2];  // x in [i0-1, i0+TX], y in [j0, j0+TY]
  float2 py[2][TY + 2][RX];  // x in [i0, i0+TX],   y in [j0-1, j0+TY]
  float2 pz[2][RY][RX];      // region
  float2 v[RY][RX];          // region, plane being formed
  float2 u[2][RY][RX];       // region, planes k and k+1
};

template <bool FIRST>
__device__ __forceinline__ void tv_load_plane(TvSmem& sm, const TvArgs& a, int k, int i0, int j0,
                                              bool load_v, bool load_pxy) {
  const int b = k & 1;
  const size_t plane = static_cast<size_t>(k) * a.ny * a.nx;
  const int tid = threadIdx.x;
  if (!FIRST) {
    if (load_pxy) {
      for (int e = tid; e < RY * (TX + 2); e += kTvThreads) {
        const int ry = e / (TX + 2), cx = e - ry * (TX + 2);
        const int gx = i0 - 1 + cx, gy = j0 + ry;
        float2 val = make_float2(0.f, 0.f);
        if (gx >= 0 && gx < a.nx && gy < a.ny) val = a.pin[0][plane + static_cast<size_t>(gy) * a.nx + gx];
        sm.px[b][ry][cx] = val;
      }
      for (int e = tid; e < (TY + 2) * RX; e += kTvThreads) {
        const int ry = e / RX, cx = e - ry * RX;
        const int gx = i0 + cx, gy = j0 - 1 + ry;
        float2 val = make_float2(0.f, 0.f);
        if (gx < a.nx && gy >= 0 && gy < a.ny) val = a.pin[1][plane + static_cast<size_t>(gy) * a.nx + gx];
        sm.py[b][ry][cx] = val;
      }
    }
    if (a.dims == 3) {
      for (int e = tid; e < RY * RX; e += kTvThreads) {
        const int ry = e / RX, cx = e - ry * RX;
        const int gx = i0 + cx, gy = j0 + ry;
        float2 val = make_float2(0.f, 0.f);
        if (gx < a.nx && gy < a.ny) val = a.pin[2][plane + static_cast<size_t>(gy) * a.nx + gx];
        sm.pz[b][ry][cx] = val;
      }
    }
  }
  if (load_v) {
    for (int e = tid; e < RY * RX; e += kTvThreads) {
      const int ry = e / RX, cx = e - ry * RX;
      const int gx = i0 + cx, gy = j0 + ry;
      float2 val = make_float2(0.f, 0.f);
      if (gx < a.nx && gy < a.ny) val = a.v[plane + static_cast<size_t>(gy) * a.nx + gx];
      sm.v[ry][cx] = val;
    }
  }
}

// u(k) over the region from the staged p (planes k and k-1) and v (plane k).
template <bool FIRST>
__device__ __forceinline__ void tv_form_u(TvSmem& sm, const TvArgs& a, int k, int i0, int j0) {
  const int b = k & 1;
  for (int e = threadIdx.x; e < RY * RX; e += kTvThreads) {
    const int ry = e / RX, cx = e - ry * RX;
    const int gx = i0 + cx, gy = j0 + ry;
    float2 u = sm.v[ry][cx];
    if (!FIRST) {
      float2 dh = make_float2(0.f, 0.f);
      if (gx >= 1) dh = cadd(dh, sm.px[b][ry][cx]);
      if (gx <= a.nx - 2) dh = csub(dh, sm.px[b][ry][cx + 1]);
      if (gy >= 1) dh = cadd(dh, sm.py[b][ry][cx]);
      if (gy <= a.ny - 2) dh = csub(dh, sm.py[b][ry + 1][cx]);
      if (a.dims == 3) {
        if (k >= 1) dh = cadd(dh, sm.pz[b ^ 1][ry][cx]);
        if (k <= a.nz - 2) dh = csub(dh, sm.pz[b][ry][cx]);
      }
      u = make_float2(u.x - a.mu * dh.x, u.y - a.mu * dh.y);
    }
    sm.u[b][ry][cx] = u;
  }
}

template <bool FIRST>
__global__ void __launch_bounds__(kTvThreads) k_tv_step(const __grid_constant__ TvArgs a) {
  __shared__ TvSmem sm;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int zc0 = blockIdx.z * a.zchunk;
  const int zc1 = min(a.nz, zc0 + a.zchunk);
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int gi = i0 + tx, gj = j0 + ty;

  // p_z of the plane below the chunk, needed by u(zc0).
  if (!FIRST && a.dims == 3 && zc0 >= 1) tv_load_plane<FIRST>(sm, a, zc0 - 1, i0, j0, false, false);
  tv_load_plane<FIRST>(sm, a, zc0, i0, j0, true, true);
  __syncthreads();
  tv_form_u<FIRST>(sm, a, zc0, i0, j0);
  __syncthreads();

  for (int k = zc0; k < zc1; ++k) {
    const bool has_next = (k + 1 < a.nz);
    if (has_next) tv_load_plane<FIRST>(sm, a, k + 1, i0, j0, true, true);
    __syncthreads();
    if (has_next) tv_form_u<FIRST>(sm, a, k + 1, i0, j0);
    __syncthreads();
    if (gi < a.nx && gj < a.ny) {
      const int b = k & 1;
      const float2 u0 = sm.u[b][ty][tx];
      float2 gx = make_float2(0.f, 0.f), gy = gx, gz = gx;
      if (gi <= a.nx - 2) gx = csub(sm.u[b][ty][tx + 1], u0);
      if (gj <= a.ny - 2) gy = csub(sm.u[b][ty + 1][tx], u0);
      if (a.dims == 3 && k <= a.nz - 2) gz = csub(sm.u[b ^ 1][ty][tx], u0);
      float2 qx, qy, qz;
      if (FIRST) {
        qx = make_float2(a.step * gx.x, a.step * gx.y);
        qy = make_float2(a.step * gy.x, a.step * gy.y);
        qz = make_float2(a.step * gz.x, a.step * gz.y);
      } else {
        const float2 ox = sm.px[b][ty][tx + 1];
        const float2 oy = sm.py[b][ty + 1][tx];
        const float2 oz = (a.dims == 3) ? sm.pz[b][ty][tx] : make_float2(0.f, 0.f);
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
  if (first)
    k_tv_step<true><<<grid, kTvThreads, 0, s>>>(a);
  else
    k_tv_step<false><<<grid, kTvThreads, 0, s>>>(a);
  return cudaGetLastError();
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
