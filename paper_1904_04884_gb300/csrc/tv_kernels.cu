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
// The TV kernels march a 32x8 x-y tile through a chunk of planes (2.5D
// blocking). Each plane of v, p_x, p_y, p_z arrives in shared memory as one
// TMA box (x from i0-2, y from j0-1 for one step or j0-2 for two: the
// stencil's halo, with the x start kept on a 16-byte boundary; out-of-range
// boxes are zero filled) into a 4-stage ring completed by mbarriers, so two planes are in flight while one is
// computed. k_tv_step2 performs two dual steps per launch (temporal blocking,
// first step recomputed on a halo ring in shared memory); k_tv_step performs
// one (for odd step counts). Outputs go out with plain coalesced stores. Every
// wait is bounded: on timeout the CTA sets the error flag, drains its copies
// in flight and exits.
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
constexpr int BW = kTvBoxW;       // TMA box: complex x in [i0-2, i0+TX+2)
constexpr int BH1 = kTvBoxH1;     //   one step:  y in [j0-1, j0+TY+1)
constexpr int BH2 = kTvBoxH2;     //   two steps: y in [j0-2, j0+TY+2)
constexpr int NSTAGE = kTvStages;
constexpr int slot_bytes(int bh) { return ((BW * bh * 8 + 127) / 128) * 128; }
constexpr int SLOT1 = slot_bytes(BH1);
constexpr int SLOT2 = slot_bytes(BH2);
constexpr int kWaitLimit = 1 << 22;   // bounded mbarrier polls before giving up

// Regions (x extent, y extent) relative to the tile origin (i0, j0):
//   A  = u of the first step:   x in [-1, TX+1], y in [-1, TY+1]
//   R2 = p of the first step:   x in [-1, TX],   y in [-1, TY]
//   R1 = u of the last step:    x in [0, TX],    y in [0, TY]
//   T  = output tile:           x in [0, TX),    y in [0, TY)
constexpr int AX = TX + 3, AY = TY + 3;
constexpr int R2X = TX + 2, R2Y = TY + 2;
constexpr int R1X = TX + 1, R1Y = TY + 1;

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

__device__ __forceinline__ float2 fma2(float2 a, float s, float2 g) {
  return make_float2(a.x + s * g.x, a.y + s * g.y);
}

// Projection of (qx, qy, qz) onto the unit ball of C^3.
__device__ __forceinline__ void project(float2& qx, float2& qy, float2& qz) {
  const float n2 = qx.x * qx.x + qx.y * qx.y + qy.x * qy.x + qy.y * qy.y + qz.x * qz.x + qz.y * qz.y;
  if (n2 > 1.f) {
    const float sc = rsqrtf(n2);
    qx.x *= sc; qx.y *= sc; qy.x *= sc; qy.y *= sc; qz.x *= sc; qz.y *= sc;
  }
}

// Plane ring fed by TMA: NSTAGE stages x 4 slots (v, p_x, p_y, p_z) of a
// BH-row box each. Plane q lives in stage (q - base) mod NSTAGE; its n-th use
// has mbarrier parity n&1.
template <int BH>
struct PlaneRing {
  static constexpr int kSlot = slot_bytes(BH);
  static constexpr int kY0 = (BH - TY) / 2;   // box row of the tile's first row
  unsigned char* smem;
  unsigned long long* bars;
  int base;
  __device__ float2 (*slot(int q, int arr) const)[BW] {
    const int s = (q - base) & (NSTAGE - 1);
    return reinterpret_cast<float2(*)[BW]>(smem + (s * 4 + arr) * kSlot);
  }
  __device__ unsigned bar(int q) const { return smem_addr(&bars[(q - base) & (NSTAGE - 1)]); }
  __device__ unsigned parity(int q) const { return static_cast<unsigned>(((q - base) / NSTAGE) & 1); }
};

template <bool FIRST, int BH>
__device__ __forceinline__ void ring_issue(const PlaneRing<BH>& r, const TvArgs& a, int q, int i0,
                                           int j0) {
  const int nslots = FIRST ? 1 : (a.dims == 3 ? 4 : 3);
  const unsigned bar = r.bar(q);
  mbar_expect_tx(bar, static_cast<unsigned>(nslots * BW * BH * 8));
  const int x = 2 * (i0 - 2), y = j0 - PlaneRing<BH>::kY0;
  tma_load_3d(smem_addr(r.slot(q, 0)), &a.tm_v, x, y, q, bar);
  if (!FIRST) {
    tma_load_3d(smem_addr(r.slot(q, 1)), &a.tm_p[0], x, y, q, bar);
    tma_load_3d(smem_addr(r.slot(q, 2)), &a.tm_p[1], x, y, q, bar);
    if (a.dims == 3) tma_load_3d(smem_addr(r.slot(q, 3)), &a.tm_p[2], x, y, q, bar);
  }
}

// Block-uniform bounded wait for plane q.
template <int BH>
__device__ __forceinline__ bool ring_wait(const PlaneRing<BH>& r, int q) {
  const bool ok = mbar_wait(r.bar(q), r.parity(q));
  return __syncthreads_and(ok) != 0;
}

// Records a failed wait and drains this CTA's copies in flight (bounded)
// before its shared memory is released.
template <int BH>
__device__ __forceinline__ void ring_abort(const PlaneRing<BH>& r, const TvArgs& a, int waited,
                                           int issued) {
  if (threadIdx.x == 0) {
    atomicExch(a.err, 1);
    for (int q = waited + 1; q <= issued; ++q) mbar_wait(r.bar(q), r.parity(q));
  }
  __syncthreads();
}

// u = v - mu D^H p at global (gx, gy) of plane k, reading the staged box at
// (by, bx) for plane k and the p_z of plane k-1 from `pzm`.
template <bool FIRST>
__device__ __forceinline__ float2 u_from_box(const TvArgs& a, float2 (*vs)[BW], float2 (*px)[BW],
                                             float2 (*py)[BW], float2 (*pz)[BW],
                                             float2 (*pzm)[BW], int by, int bx, int gx, int gy,
                                             int k) {
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
  return uu;
}

struct TvLayout1 {   // one dual step per launch
  static constexpr int kUBytes = 2 * R1Y * R1X * 8;
  static constexpr int kBarOffset = NSTAGE * 4 * SLOT1 + kUBytes;
  static constexpr int kBytes = kBarOffset + NSTAGE * 8;
};

// One dual gradient-projection step (used for an odd step count).
template <bool FIRST>
__global__ void __launch_bounds__(kTvThreads) k_tv_step(const __grid_constant__ TvArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  float2(*U)[R1Y][R1X] = reinterpret_cast<float2(*)[R1Y][R1X]>(smem + NSTAGE * 4 * SLOT1);
  PlaneRing<BH1> ring{smem, reinterpret_cast<unsigned long long*>(smem + TvLayout1::kBarOffset),
                      static_cast<int>(blockIdx.z) * a.zchunk - 1};
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int zc0 = blockIdx.z * a.zchunk;
  const int zc1 = min(a.nz, zc0 + a.zchunk);
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int gi = i0 + tx, gj = j0 + ty;
  const int qlast = min(zc1, a.nz - 1);

  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) mbar_init(smem_addr(&ring.bars[s]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0)
    for (int q = ring.base; q < ring.base + NSTAGE && q <= qlast; ++q) ring_issue<FIRST>(ring, a, q, i0, j0);
  int issued = min(ring.base + NSTAGE - 1, qlast);
  int waited = ring.base - 1;

  auto form_u = [&](int k) {
    float2(*u)[R1X] = U[k & 1];
    for (int e = tid; e < R1Y * R1X; e += kTvThreads) {
      const int ry = e / R1X, rx = e - ry * R1X;
      u[ry][rx] = u_from_box<FIRST>(a, ring.slot(k, 0), ring.slot(k, 1), ring.slot(k, 2),
                                    ring.slot(k, 3), ring.slot(k - 1, 3), ry + 1, rx + 2, i0 + rx,
                                    j0 + ry, k);
    }
  };

  if (!ring_wait(ring, ring.base)) { ring_abort(ring, a, waited, issued); return; }
  waited = ring.base;
  if (!ring_wait(ring, zc0)) { ring_abort(ring, a, waited, issued); return; }
  waited = zc0;
  form_u(zc0);
  __syncthreads();

  for (int k = zc0; k < zc1; ++k) {
    if (k + 3 <= qlast) {     // stage of plane k-1 is free
      if (tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        ring_issue<FIRST>(ring, a, k + 3, i0, j0);
      }
      issued = k + 3;
    }
    const bool has_next = (k + 1 < a.nz);
    if (has_next) {
      if (!ring_wait(ring, k + 1)) { ring_abort(ring, a, waited, issued); return; }
      waited = k + 1;
      form_u(k + 1);
    }
    __syncthreads();
    if (gi < a.nx && gj < a.ny) {
      float2(*u)[R1X] = U[k & 1];
      float2(*un)[R1X] = U[(k + 1) & 1];
      const float2 u0 = u[ty][tx];
      float2 gx = make_float2(0.f, 0.f), gy = gx, gz = gx;
      if (gi <= a.nx - 2) gx = csub(u[ty][tx + 1], u0);
      if (gj <= a.ny - 2) gy = csub(u[ty + 1][tx], u0);
      if (a.dims == 3 && k <= a.nz - 2) gz = csub(un[ty][tx], u0);
      float2 qx = make_float2(0.f, 0.f), qy = qx, qz = qx;
      if (!FIRST) {
        qx = ring.slot(k, 1)[ty + 1][tx + 2];
        qy = ring.slot(k, 2)[ty + 1][tx + 2];
        if (a.dims == 3) qz = ring.slot(k, 3)[ty + 1][tx + 2];
      }
      qx = fma2(qx, a.step, gx);
      qy = fma2(qy, a.step, gy);
      qz = fma2(qz, a.step, gz);
      project(qx, qy, qz);
      const size_t gidx = (static_cast<size_t>(k) * a.ny + gj) * a.nx + gi;
      a.pout[0][gidx] = qx;
      a.pout[1][gidx] = qy;
      if (a.dims == 3) a.pout[2][gidx] = qz;
    }
    __syncthreads();
  }
}

struct TvLayout2 {   // two dual steps per launch
  static constexpr int kU0Off = NSTAGE * 4 * SLOT2;
  static constexpr int kU0Bytes = 2 * AY * AX * 8;
  static constexpr int kP1Off = kU0Off + kU0Bytes;
  static constexpr int kP1Bytes = 2 * 3 * R2Y * R2X * 8;
  static constexpr int kU1Off = kP1Off + kP1Bytes;
  static constexpr int kU1Bytes = 2 * R1Y * R1X * 8;
  static constexpr int kBarOffset = kU1Off + kU1Bytes;
  static constexpr int kBytes = kBarOffset + NSTAGE * 8;
};

// Two dual gradient-projection steps per launch (temporal blocking). With p^0
// the input dual and p^2 the output, per plane tick t of the z march:
//   (a) u^0(t+1) over A   from p^0(t+1), p^0_z(t), v(t+1)   [TMA ring]
//   (b) p^1(t)   over R2  from u^0(t), u^0(t+1), p^0(t)
//   (c) u^1(t)   over R1  from p^1(t), p^1_z(t-1), v(t)
//   (d) p^2(t-1) over T   from u^1(t-1), u^1(t), p^1(t-1)   -> global
// Step 1 is recomputed on a one-voxel halo ring around the tile (R2), which
// needs a two-voxel halo of p^0 and v: the TMA box covers x in [i0-2, i0+TX+2)
// and y in [j0-2, j0+TY+2). HBM traffic per voxel for two steps is one read of
// v and p^0 and one write of p^2.
template <bool FIRST>
__global__ void __launch_bounds__(kTvThreads, 2) k_tv_step2(const __grid_constant__ TvArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  float2(*U0)[AY][AX] = reinterpret_cast<float2(*)[AY][AX]>(smem + TvLayout2::kU0Off);
  float2(*P1)[3][R2Y][R2X] = reinterpret_cast<float2(*)[3][R2Y][R2X]>(smem + TvLayout2::kP1Off);
  float2(*U1)[R1Y][R1X] = reinterpret_cast<float2(*)[R1Y][R1X]>(smem + TvLayout2::kU1Off);
  const int zc0 = blockIdx.z * a.zchunk;
  const int zc1 = min(a.nz, zc0 + a.zchunk);
  // planes zc0-2 .. zc1+1 are read (out-of-range planes arrive zero filled)
  PlaneRing<BH2> ring{smem, reinterpret_cast<unsigned long long*>(smem + TvLayout2::kBarOffset),
                      zc0 - 2};
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int tid = threadIdx.x;
  const int qlast = zc1 + 1;

  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) mbar_init(smem_addr(&ring.bars[s]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0)
    for (int q = ring.base; q < ring.base + NSTAGE && q <= qlast; ++q) ring_issue<FIRST>(ring, a, q, i0, j0);
  int issued = min(ring.base + NSTAGE - 1, qlast);
  int waited = ring.base - 1;

  // (a) u^0(q) over A (box coordinates: A origin is box (1, 1))
  auto step_a = [&](int q) {
    float2(*u)[AX] = U0[q & 1];
    for (int e = tid; e < AY * AX; e += kTvThreads) {
      const int ry = e / AX, rx = e - ry * AX;
      u[ry][rx] = u_from_box<FIRST>(a, ring.slot(q, 0), ring.slot(q, 1), ring.slot(q, 2),
                                    ring.slot(q, 3), ring.slot(q - 1, 3), ry + 1, rx + 1,
                                    i0 - 1 + rx, j0 - 1 + ry, q);
    }
  };
  // (b) p^1(q) over R2 (R2 origin is A (0, 0) and box (1, 1))
  auto step_b = [&](int q) {
    float2(*u)[AX] = U0[q & 1];
    float2(*un)[AX] = U0[(q + 1) & 1];
    float2(*p1)[R2Y][R2X] = P1[q & 1];
    for (int e = tid; e < R2Y * R2X; e += kTvThreads) {
      const int ry = e / R2X, rx = e - ry * R2X;
      const int gx = i0 - 1 + rx, gy = j0 - 1 + ry;
      const float2 u0 = u[ry][rx];
      float2 dx = make_float2(0.f, 0.f), dy = dx, dz = dx;
      if (gx <= a.nx - 2) dx = csub(u[ry][rx + 1], u0);
      if (gy <= a.ny - 2) dy = csub(u[ry + 1][rx], u0);
      if (a.dims == 3 && q <= a.nz - 2) dz = csub(un[ry][rx], u0);
      float2 qx = make_float2(0.f, 0.f), qy = qx, qz = qx;
      if (!FIRST) {
        qx = ring.slot(q, 1)[ry + 1][rx + 1];
        qy = ring.slot(q, 2)[ry + 1][rx + 1];
        if (a.dims == 3) qz = ring.slot(q, 3)[ry + 1][rx + 1];
      }
      qx = fma2(qx, a.step, dx);
      qy = fma2(qy, a.step, dy);
      qz = fma2(qz, a.step, dz);
      project(qx, qy, qz);
      p1[0][ry][rx] = qx;
      p1[1][ry][rx] = qy;
      p1[2][ry][rx] = qz;
    }
  };
  // (c) u^1(q) over R1 (R1 origin is R2 (1, 1) and box (2, 2))
  auto step_c = [&](int q) {
    float2(*p1)[R2Y][R2X] = P1[q & 1];
    float2(*p1m)[R2Y][R2X] = P1[(q + 1) & 1];   // plane q-1
    float2(*vs)[BW] = ring.slot(q, 0);
    float2(*u)[R1X] = U1[q & 1];
    for (int e = tid; e < R1Y * R1X; e += kTvThreads) {
      const int ry = e / R1X, rx = e - ry * R1X;
      const int gx = i0 + rx, gy = j0 + ry;
      float2 dh = make_float2(0.f, 0.f);
      if (gx >= 1) dh = cadd(dh, p1[0][ry + 1][rx]);
      if (gx <= a.nx - 2) dh = csub(dh, p1[0][ry + 1][rx + 1]);
      if (gy >= 1) dh = cadd(dh, p1[1][ry][rx + 1]);
      if (gy <= a.ny - 2) dh = csub(dh, p1[1][ry + 1][rx + 1]);
      if (a.dims == 3) {
        if (q >= 1) dh = cadd(dh, p1m[2][ry + 1][rx + 1]);
        if (q <= a.nz - 2) dh = csub(dh, p1[2][ry + 1][rx + 1]);
      }
      const float2 v = vs[ry + 2][rx + 2];
      u[ry][rx] = make_float2(v.x - a.mu * dh.x, v.y - a.mu * dh.y);
    }
  };
  // (d) p^2(q) over the tile -> global
  auto step_d = [&](int q) {
    const int tx = tid % TX, ty = tid / TX;
    const int gi = i0 + tx, gj = j0 + ty;
    if (gi >= a.nx || gj >= a.ny) return;
    float2(*u)[R1X] = U1[q & 1];
    float2(*un)[R1X] = U1[(q + 1) & 1];
    float2(*p1)[R2Y][R2X] = P1[q & 1];
    const float2 u0 = u[ty][tx];
    float2 dx = make_float2(0.f, 0.f), dy = dx, dz = dx;
    if (gi <= a.nx - 2) dx = csub(u[ty][tx + 1], u0);
    if (gj <= a.ny - 2) dy = csub(u[ty + 1][tx], u0);
    if (a.dims == 3 && q <= a.nz - 2) dz = csub(un[ty][tx], u0);
    float2 qx = fma2(p1[0][ty + 1][tx + 1], a.step, dx);
    float2 qy = fma2(p1[1][ty + 1][tx + 1], a.step, dy);
    float2 qz = fma2(p1[2][ty + 1][tx + 1], a.step, dz);
    project(qx, qy, qz);
    const size_t gidx = (static_cast<size_t>(q) * a.ny + gj) * a.nx + gi;
    a.pout[0][gidx] = qx;
    a.pout[1][gidx] = qy;
    if (a.dims == 3) a.pout[2][gidx] = qz;
  };

  // pre-tick: u^0(zc0-1) needs planes zc0-2 (p_z) and zc0-1
  if (!ring_wait(ring, zc0 - 2)) { ring_abort(ring, a, waited, issued); return; }
  waited = zc0 - 2;
  if (!ring_wait(ring, zc0 - 1)) { ring_abort(ring, a, waited, issued); return; }
  waited = zc0 - 1;
  step_a(zc0 - 1);
  __syncthreads();

  for (int t = zc0 - 1; t <= zc1; ++t) {
    // stage of plane t-1 is free from tick t on: refill it with plane t+3
    if (t + 3 <= qlast) {
      if (tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        ring_issue<FIRST>(ring, a, t + 3, i0, j0);
      }
      issued = t + 3;
    }
    if (!ring_wait(ring, t + 1)) { ring_abort(ring, a, waited, issued); return; }
    waited = t + 1;
    step_a(t + 1);
    __syncthreads();
    step_b(t);
    __syncthreads();
    if (t >= zc0) {
      step_c(t);
      __syncthreads();
      if (t >= zc0 + 1) step_d(t - 1);
      __syncthreads();
    }
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

cudaError_t launch_tv_step(bool first, int nsteps, const TvArgs& a, cudaStream_t s) {
  dim3 grid((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY, (a.nz + a.zchunk - 1) / a.zchunk);
  auto kern = nsteps == 2 ? (first ? k_tv_step2<true> : k_tv_step2<false>)
                          : (first ? k_tv_step<true> : k_tv_step<false>);
  const int bytes = nsteps == 2 ? TvLayout2::kBytes : TvLayout1::kBytes;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  kern<<<grid, kTvThreads, bytes, s>>>(a);
  return cudaGetLastError();
}

// 3D tensor map over a complex64 volume viewed as float32 [nz][ny][2 nx], box
// of box_rows rows x 2 kTvBoxW floats x 1 plane, zero fill out of bounds.
cudaError_t make_volume_tmap(CUtensorMap* tm, const void* base, int nx, int ny, int nz,
                             int box_rows) {
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
  const cuuint32_t box[3] = {2 * kTvBoxW, static_cast<cuuint32_t>(box_rows), 1};
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
