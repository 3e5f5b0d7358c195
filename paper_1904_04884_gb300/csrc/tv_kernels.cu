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
// The TV kernels stream an x-y tile through a chunk of planes (2.5D
// blocking). Each plane of v, p_x, p_y, p_z arrives in shared memory as one
// TMA box (the stencil's halo included, its x start kept on a 16-byte
// boundary; out-of-range boxes are zero filled) in a ring of stages completed
// by mbarriers, so that planes are in flight while one is computed.
//   k_tv_step:  one dual step, 32 x 8 tile, one thread per position, 4 stages.
//   k_tv_step2: two dual steps per launch (temporal blocking: the first step
//               recomputed on a one-voxel halo ring), one warp per tile row,
//               two x positions per lane, 60 x 16 tile, 3 stages. Its FINAL
//               form (58 x 11 tile, one more halo ring) also forms
//               x = soft(v - mu D^H p^2) and, for FISTA, y_{k+1} and the
//               restart product, so the last dual field never reaches memory.
// An odd step count starts with one k_tv_step launch. Outputs go out with
// plain coalesced stores. Every wait is bounded: on timeout the CTA sets the
// error flag, drains its copies in flight (bounded) and exits.
//
// The separate finalize kernel (used when the finalize is not fused) forms
// u = v - mu D^H p, soft-thresholds it, and in FISTA mode writes x_k and
// y_{k+1} = x_k + beta (x_k - x_{k-1}) and reduces the gradient-restart
// inner product Re<y_k - x_k, x_k - x_{k-1}> (FP32 over 8 voxels, FP64
// above). The last block of the grid (ticket counter) updates t, beta and the
// restart flag on the device, so no scalar crosses to the host.
#include <cuda_runtime.h>

#include <algorithm>

#include "rihv_internal.cuh"

namespace rihv {
namespace {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

constexpr int TX = kTvTx;
constexpr int TY = kTvTy;
constexpr int BW = kTvBoxW;       // one-step TMA box: complex x in [i0-2, i0+TX+2)
constexpr int BH1 = kTvBoxH1;     //                   y in [j0-1, j0+TY+1)
constexpr int NSTAGE = kTvStages;
constexpr int slot_bytes(int bw, int bh) { return ((bw * bh * 8 + 127) / 128) * 128; }
constexpr int SLOT1 = slot_bytes(BW, BH1);
constexpr int kWaitLimit = 1 << 22;   // bounded mbarrier polls before giving up

// One-step kernel: u = v - mu D^H p is formed on the tile plus one column and
// one row (x in [0, TX], y in [0, TY] relative to the tile origin), the region
// whose forward differences the tile's p update reads.
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
// Bounded wait: true if the phase completed, false after `limit` polls.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, int limit = kWaitLimit) {
  for (int it = 0; it < limit; ++it)
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

// Plane ring fed by TMA: NS stages x 4 slots (v, p_x, p_y, p_z) of a
// BH x BWR box each. Plane q lives in stage (q - base) mod NS; its n-th use
// has mbarrier parity n&1.
template <int BWR, int BH, int Y0, int NS, int X0 = 2>
struct PlaneRing {
  static constexpr int kSlot = slot_bytes(BWR, BH);
  static constexpr int kW = BWR;
  static constexpr int kH = BH;
  static constexpr int kY0 = Y0;   // box row of the tile's first row
  static constexpr int kX0 = X0;   // box column of the tile's first column
  unsigned char* smem;
  unsigned long long* bars;
  int base;                        // first plane of the ring (q - base >= 0)
  __device__ int stage(int q) const { return static_cast<int>(static_cast<unsigned>(q - base) % NS); }
  __device__ float2 (*slot(int q, int arr) const)[BWR] {
    return reinterpret_cast<float2(*)[BWR]>(smem + (stage(q) * 4 + arr) * kSlot);
  }
  __device__ unsigned bar(int q) const { return smem_addr(&bars[stage(q)]); }
  __device__ unsigned parity(int q) const {
    return (static_cast<unsigned>(q - base) / NS) & 1u;
  }
};

template <bool FIRST, class Ring>
__device__ __forceinline__ void ring_issue(const Ring& r, const TvArgs& a, int q, int i0, int j0) {
  const int nslots = FIRST ? 1 : (a.dims == 3 ? 4 : 3);
  const unsigned bar = r.bar(q);
  mbar_expect_tx(bar, static_cast<unsigned>(nslots * Ring::kW * Ring::kH * 8));
  const int x = 2 * (i0 - Ring::kX0), y = j0 - Ring::kY0;
  tma_load_3d(smem_addr(r.slot(q, 0)), &a.tm_v, x, y, q, bar);
  if (!FIRST) {
    tma_load_3d(smem_addr(r.slot(q, 1)), &a.tm_p[0], x, y, q, bar);
    tma_load_3d(smem_addr(r.slot(q, 2)), &a.tm_p[1], x, y, q, bar);
    if (a.dims == 3) tma_load_3d(smem_addr(r.slot(q, 3)), &a.tm_p[2], x, y, q, bar);
  }
}

// Block-uniform bounded wait for plane q.
template <class Ring>
__device__ __forceinline__ bool ring_wait(const Ring& r, int q) {
  const bool ok = mbar_wait(r.bar(q), r.parity(q));
  return __syncthreads_and(ok) != 0;
}

// Records a failed wait and drains this CTA's copies in flight (bounded)
// before its shared memory is released.
template <class Ring>
__device__ __forceinline__ void ring_abort(const Ring& r, const TvArgs& a, int waited,
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

// One dual gradient-projection step (used for an odd step count). FGP: the
// step of the accelerated dual, which also writes the extrapolated dual for
// the next step (see TvArgs).
template <bool FIRST, bool FGP = false>
__global__ void __launch_bounds__(kTvThreads) k_tv_step(const __grid_constant__ TvArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  float2(*U)[R1Y][R1X] = reinterpret_cast<float2(*)[R1Y][R1X]>(smem + NSTAGE * 4 * SLOT1);
  PlaneRing<BW, BH1, 1, NSTAGE> ring{smem, reinterpret_cast<unsigned long long*>(smem + TvLayout1::kBarOffset),
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
      if (FGP && a.rout[0]) {
        // r_{k+1} = p_k + beta (p_k - p_{k-1}), p_0 = 0
        float2 ox = make_float2(0.f, 0.f), oy = ox, oz = ox;
        if (!FIRST) {
          ox = a.pprev[0][gidx];
          oy = a.pprev[1][gidx];
          if (a.dims == 3) oz = a.pprev[2][gidx];
        }
        const float bt = a.fgp_beta;
        a.rout[0][gidx] = make_float2(qx.x + bt * (qx.x - ox.x), qx.y + bt * (qx.y - ox.y));
        a.rout[1][gidx] = make_float2(qy.x + bt * (qy.x - oy.x), qy.y + bt * (qy.y - oy.y));
        if (a.dims == 3)
          a.rout[2][gidx] = make_float2(qz.x + bt * (qz.x - oz.x), qz.y + bt * (qz.y - oz.y));
      }
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

// Reciprocal square root by the hardware approximation (PTX rsqrt.approx,
// relative error below 2^-22; inputs here are > 1 or > kappa^2, never
// subnormal, so flushing subnormals changes nothing).
__device__ __forceinline__ float rsqrt_hw(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// The shrinkage through the reciprocal square root (one hardware
// approximation instead of a square root and a division).
__device__ __forceinline__ float2 soft_rsqrt(float2 u, float kappa) {
  const float m2 = u.x * u.x + u.y * u.y;
  const float s = (m2 > kappa * kappa) ? (1.f - kappa * rsqrt_hw(m2)) : 0.f;
  return make_float2(u.x * s, u.y * s);
}

__device__ __forceinline__ float2 soft(float2 u, float kappa) {
  const float mag = sqrtf(u.x * u.x + u.y * u.y);
  const float s = (mag > kappa) ? (1.f - kappa / mag) : 0.f;
  return make_float2(u.x * s, u.y * s);
}


// FISTA scalars after the finalize of iteration k, from the restart inner
// product Re<y_k - x_k, x_k - x_{k-1}> (O'Donoghue-Candes gradient restart):
// t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2, or 1 on restart; beta for the next
// extrapolation from t_{k+1} and t_{k+2}.
__device__ __forceinline__ void fista_update(DevScalars* sc, double dot) {
  sc->beta_used = sc->beta;
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
}

constexpr int TX2 = kTv2Tx;
template <int NW>
struct TvLayout2 {   // two dual steps per launch, NW warps (one per halo row)
  static constexpr int kSlot = slot_bytes(kTv2BoxW, NW + 1);
  static constexpr int kXOff = kTv2Stages * 4 * kSlot;
  // exchange rows for y-neighbours (one pair of complex values per lane),
  // double buffered by plane parity: u0, p1_y, u1 and (fused finalize) p2_y,
  // each [2][NW][32]
  static constexpr int kXRow = NW * 32 * 16;
  static constexpr int kBarOffset = kXOff + 8 * kXRow;
  static constexpr int kBytes = kBarOffset + kTv2Stages * 8;
};

// Packed two-lane FP32 arithmetic (f32x2, sm_100 and later) on complex
// values: one instruction per complex subtract, multiply-add or scale,
// each lane rounded as the scalar instruction would.
__device__ __forceinline__ unsigned long long as_b64(float2 a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ float2 as_f2(unsigned long long r) {
  float2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
__device__ __forceinline__ float2 x2sub(float2 a, float2 b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(as_b64(a)), "l"(as_b64(b)));
  return as_f2(d);
}
__device__ __forceinline__ float2 x2mul(float2 a, float2 b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(as_b64(a)), "l"(as_b64(b)));
  return as_f2(d);
}
// a * b + c, lane by lane, one rounding
__device__ __forceinline__ float2 x2fma(float2 a, float2 b, float2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(as_b64(a)), "l"(as_b64(b)), "l"(as_b64(c)));
  return as_f2(d);
}
// Projection onto the unit ball of C^3 with packed arithmetic, branch free
// (a scale of 1 leaves the vector unchanged).
__device__ __forceinline__ void project2(float2& qx, float2& qy, float2& qz) {
  const float2 s = x2fma(qz, qz, x2fma(qy, qy, x2mul(qx, qx)));
  const float n2 = s.x + s.y;
  const float r = n2 > 1.f ? rsqrt_hw(n2) : 1.f;
  const float2 sc = make_float2(r, r);
  qx = x2mul(qx, sc);
  qy = x2mul(qy, sc);
  qz = x2mul(qz, sc);
}
__device__ __forceinline__ float2 splat(float v) { return make_float2(v, v); }

__device__ __forceinline__ float2 shfl_up2(float2 v) {
  return make_float2(__shfl_up_sync(0xffffffffu, v.x, 1), __shfl_up_sync(0xffffffffu, v.y, 1));
}

// Adds v to the compensated sum (hi, lo) (Knuth's TwoSum: the rounding error
// of hi + v goes to lo).
__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float v) {
  const float s = hi + v;
  const float b = s - hi;
  lo += (hi - (s - b)) + (v - b);
  hi = s;
}

__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float4 pack4(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }

// Two dual gradient-projection steps per launch (temporal blocking). With p^0
// the input dual and p^2 the output, a 60 x 16 tile marches through its chunk
// of planes. Thread (warp w, lane l) owns the two positions x = i0-2+2l+e
// (e = 0, 1), y = j0-1+w of the halo (19 rows x 64 columns) and, per plane
// tick t, computes
//   (a) u^0(t+1) = v - mu D^H p^0              [staged box of plane t+1]
//   (b) p^1(t)   = Pi(p^0 + step D u^0)        [u^0(t), u^0(t+1)]
//   (c) u^1(t)   = v - mu D^H p^1              [p^1(t), p^1_z(t-1)]
//   (d) p^2(t-1) = Pi(p^1 + step D u^1)        [u^1(t-1), u^1(t)] -> global
// z-neighbours stay in registers across ticks; x-neighbours are the thread's
// other position, or the neighbouring lane's (a shuffle or the exchange row);
// y-neighbours pass through shared-memory exchange rows, double buffered by
// plane parity. One barrier per tick, between (b) and (c), orders every
// exchange: a row written before barrier k is read after it and rewritten
// only after barrier k+1; it also carries the vote on the ring wait. Step 1
// is recomputed on the halo ring, so each voxel's v and p^0 are read from HBM
// about once and p^2 written once for two steps. Positions outside a step's
// region compute values that no output uses; every use is guarded by the same
// global-index boundary conditions as the single step. Needs nx even (pairs
// of outputs are stored as 16-byte words).
//
// FINAL (the last launch of a prox): the tile is 58 x 11 (15 warps) and the
// halo one voxel wider on the low sides (x = i0-4+2l+e, y = j0-2+w, one more
// plane before the chunk), so that p^2 is known at x-1, y-1 and z-1 of every
// tile voxel; after a second barrier per tick,
//   (e) x(t-1) = soft(v - mu D^H p^2, kappa)   [p^2(t-1), p^2_z(t-2)]
// is written instead of p^2, in FISTA mode with y_{k+1} = x + beta (x -
// x_prev) and the restart inner product, reduced like the finalize kernel.
// FMODE: FIN_PROX, FIN_FISTA, or kFinFistaOcc (FISTA that also records
// which planes hold a non-zero voxel, for the empty-plane skip).
template <bool FIRST, bool FINAL, int FMODE = FIN_PROX>
__global__ void __launch_bounds__(32 * (FINAL ? kTv2WarpsF : kTv2Warps), 1)
    k_tv_step2(const __grid_constant__ TvArgs a) {
  constexpr bool FISTA = FINAL && (FMODE == FIN_FISTA || FMODE == kFinFistaOcc);
  constexpr bool OCC = FINAL && FMODE == kFinFistaOcc;
  constexpr int TXk = FINAL ? kTv2TxF : kTv2Tx;
  constexpr int TYk = FINAL ? kTv2TyF : kTv2Ty;
  constexpr int NW2 = FINAL ? kTv2WarpsF : kTv2Warps;
  using Layout = TvLayout2<NW2>;
  constexpr int X0 = FINAL ? 4 : 2;    // box and lane 0 start at x = i0 - X0
  constexpr int Y0 = FINAL ? 3 : 2;    // box starts at y = j0 - Y0, warp 0 at j0 - Y0 + 1
  constexpr int L = FINAL ? 1 : 0;     // extra planes of z halo before the chunk
  using Ring = PlaneRing<kTv2BoxW, NW2 + 1, Y0, kTv2Stages, X0>;
  extern __shared__ __align__(128) unsigned char smem[];
  using Row = float4[NW2][32];
  using Box4 = const float4(*)[kTv2BoxW / 2];
  Row* XU0 = reinterpret_cast<Row*>(smem + Layout::kXOff);
  Row* XP1 = XU0 + 2;
  Row* XU1 = XU0 + 4;
  Row* XP2 = XU0 + 6;                           // FINAL only
  // CTA -> (tile, z-chunk), 1D grid: tiles [0, ka) in z-chunks of zchunk
  // planes, then tiles [ka, ntiles) in z-chunks of zchunk2, chunk-major within
  // each part (x-adjacent tiles launch together). Without a split this is the
  // order of an (x tiles, y tiles, z-chunks) grid.
  const int tiles_x = (a.nx + TXk - 1) / TXk;
  const int ntiles = tiles_x * ((a.ny + TYk - 1) / TYk);
  const int ka = a.zchunk2 > 0 ? min(a.split_tile, ntiles) : ntiles;
  const int ctas_a = ka * ((a.nz + a.zchunk - 1) / a.zchunk);
  int tile, zc0, zc1;
  if (static_cast<int>(blockIdx.x) < ctas_a) {
    tile = blockIdx.x % ka;
    zc0 = (blockIdx.x / ka) * a.zchunk;
    zc1 = min(a.nz, zc0 + a.zchunk);
  } else {
    const int b2 = blockIdx.x - ctas_a, kb = ntiles - ka;
    tile = ka + b2 % kb;
    zc0 = (b2 / kb) * a.zchunk2;
    zc1 = min(a.nz, zc0 + a.zchunk2);
  }
  Ring ring{smem, reinterpret_cast<unsigned long long*>(smem + Layout::kBarOffset), zc0 - 2 - L};
  const int i0 = (tile % tiles_x) * TXk, j0 = (tile / tiles_x) * TYk;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int gx0 = i0 - X0 + 2 * lane, gy = j0 - (Y0 - 1) + w;   // element e at x = gx0 + e
  const int by = w + 1;                                 // own row in the box
  const int cm = lane > 0 ? 2 * lane - 1 : 0;           // box column x-1 of element 0
  const int ln = lane < 31 ? lane + 1 : lane;           // next lane (x+1 of element 1)
  const int qlast = zc1 + 1;
  const bool out_pair = w >= Y0 - 1 && w <= Y0 - 2 + TYk && lane >= X0 / 2 &&
                        lane <= (TXk + X0 - 2) / 2 && gx0 < a.nx && gy < a.ny;
  const int wn = w + 1 < NW2 ? w + 1 : w;       // y+1 row (the last row's value is unused)
  const int wp = w >= 1 ? w - 1 : w;            // y-1 row (the first row's value is unused)
  // Boundary conditions as multipliers, so that every term is one packed
  // multiply-add: m_lo = 1 where the backward neighbour exists (D^H term
  // +p(x-1)), m_hi = -1 where the forward difference exists (D^H term -p(x)),
  // s_hi = step there (the step's D u term); 0 elsewhere. Adding or
  // subtracting through an exact +-1 or 0 multiplier rounds as the add itself.
  // With gx0 and nx even, element 0 always has a forward neighbour and
  // element 1 a backward one inside the volume; the exceptions lie outside it
  // (x = -1, x >= nx), where values are computed but never used.
  const float2 mxlo0 = splat(gx0 >= 1 ? 1.f : 0.f);
  const float2 mxhi1 = splat(gx0 + 1 <= a.nx - 2 ? -1.f : 0.f);
  const float2 sxhi1 = splat(gx0 + 1 <= a.nx - 2 ? a.step : 0.f);
  const float2 stp = splat(a.step);
  const float2 mylo = splat(gy >= 1 ? 1.f : 0.f);
  const float2 myhi = splat(gy <= a.ny - 2 ? -1.f : 0.f);
  const float2 syhi = splat(gy <= a.ny - 2 ? a.step : 0.f);
  const float2 nmu = splat(-a.mu);

  // OCC: which planes of the chunk hold a non-zero voxel of x_k or y_{k+1}
  __shared__ unsigned char occ_s[OCC ? kTvMaxChunk : 1];
  if (OCC)
    for (int q = tid; q < kTvMaxChunk; q += blockDim.x) occ_s[q] = 0;
  if (tid == 0) {
    for (int s = 0; s < kTv2Stages; ++s) mbar_init(smem_addr(&ring.bars[s]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0)
    for (int q = ring.base; q < ring.base + kTv2Stages && q <= qlast; ++q)
      ring_issue<FIRST>(ring, a, q, i0, j0);
  int issued = min(ring.base + kTv2Stages - 1, qlast);
  int waited = ring.base - 1;

  const float2 zero = make_float2(0.f, 0.f);
  // per-position state of plane t (index e = element)
  float2 u0_t[2] = {zero, zero}, v_t[2] = {zero, zero};
  float2 p0_t[3][2] = {{zero, zero}, {zero, zero}, {zero, zero}};
  float2 p1_prev[3][2] = {{zero, zero}, {zero, zero}, {zero, zero}};
  float2 p1_t[3][2] = {{zero, zero}, {zero, zero}, {zero, zero}};
  float2 u1_prev[2] = {zero, zero}, u1_t[2] = {zero, zero};
  // FINAL: v of plane t-1 and p^2_z of plane t-2; FISTA restart partials
  float2 v_prev[2] = {zero, zero}, p2z_prev[2] = {zero, zero};
  float dot_hi = 0.f, dot_lo = 0.f;   // compensated FP32 sum of the restart product
  const float beta = FISTA ? static_cast<float>(a.sc->beta) : 0.f;

  // prologue: p^0_z of the ring's first plane (read by u^0 of the next)
  if (!ring_wait(ring, ring.base)) { ring_abort(ring, a, waited, issued); return; }
  waited = ring.base;
  if (!FIRST && a.dims == 3) {
    const float4 pz = reinterpret_cast<Box4>(ring.slot(ring.base, 3))[by][lane];
    p0_t[2][0] = lo2(pz);
    p0_t[2][1] = hi2(pz);
  }
  __syncthreads();

  for (int t = ring.base; t <= zc1; ++t) {
    // plane t was last read in tick t-1, before that tick's barrier: refill
    // its stage with plane t+NS
    if (t + kTv2Stages <= qlast) {
      if (tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        ring_issue<FIRST>(ring, a, t + kTv2Stages, i0, j0);
      }
      issued = t + kTv2Stages;
    }
    // FINAL + FISTA: x_{k-1} and y_k of plane t-1 are loaded now, a whole
    // tick before step (e) uses them
    float4 xp4 = make_float4(0.f, 0.f, 0.f, 0.f), yk4 = xp4;
    if (FISTA && t >= zc0 + 1 && out_pair) {
      const size_t gidx = (static_cast<size_t>(t - 1) * a.ny + gy) * a.nx + gx0;
      xp4 = *reinterpret_cast<const float4*>(a.x_prev + gidx);
      yk4 = *reinterpret_cast<const float4*>(a.y + gidx);
    }
    // (a) u^0(t+1) from the box of plane t+1 (the wait is voted on below)
    const int q = t + 1;
    const bool ok = mbar_wait(ring.bar(q), ring.parity(q));
    float2 v_n[2], p0_n[3][2] = {{zero, zero}, {zero, zero}, {zero, zero}}, u0_n[2];
    {
      const float4 vv = reinterpret_cast<Box4>(ring.slot(q, 0))[by][lane];
      v_n[0] = lo2(vv);
      v_n[1] = hi2(vv);
      u0_n[0] = v_n[0];
      u0_n[1] = v_n[1];
      if (!FIRST) {
        float2(*px)[kTv2BoxW] = ring.slot(q, 1);
        float2(*py)[kTv2BoxW] = ring.slot(q, 2);
        const float4 px4 = reinterpret_cast<Box4>(px)[by][lane];
        const float4 py4 = reinterpret_cast<Box4>(py)[by][lane];
        const float4 pym4 = reinterpret_cast<Box4>(py)[by - 1][lane];
        const float2 pxm0 = px[by][cm];
        p0_n[0][0] = lo2(px4);
        p0_n[0][1] = hi2(px4);
        p0_n[1][0] = lo2(py4);
        p0_n[1][1] = hi2(py4);
        float2 mzlo = zero, mzhi = zero;
        if (a.dims == 3) {
          const float4 pz4 = reinterpret_cast<Box4>(ring.slot(q, 3))[by][lane];
          p0_n[2][0] = lo2(pz4);
          p0_n[2][1] = hi2(pz4);
          mzlo = splat(q >= 1 ? 1.f : 0.f);
          mzhi = splat(q <= a.nz - 2 ? -1.f : 0.f);
        }
        const float2 pxm[2] = {pxm0, p0_n[0][0]};
        const float2 pym[2] = {lo2(pym4), hi2(pym4)};
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          float2 dh = e == 0 ? x2mul(mxlo0, pxm[0]) : pxm[1];
          dh = e == 0 ? x2sub(dh, p0_n[0][0]) : x2fma(mxhi1, p0_n[0][1], dh);
          dh = x2fma(mylo, pym[e], dh);
          dh = x2fma(myhi, p0_n[1][e], dh);
          if (a.dims == 3) {
            dh = x2fma(mzlo, p0_t[2][e], dh);
            dh = x2fma(mzhi, p0_n[2][e], dh);
          }
          u0_n[e] = x2fma(nmu, dh, v_n[e]);
        }
      }
      XU0[q & 1][w][lane] = pack4(u0_n[0], u0_n[1]);
    }
    // (b) p^1(t)
    if (t >= zc0 - 1 - L) {
      const float2 ux[2] = {u0_t[1], lo2(XU0[t & 1][w][ln])};
      const float4 uy4 = XU0[t & 1][wn][lane];
      const float2 uy[2] = {lo2(uy4), hi2(uy4)};
      const float2 szhi = splat(a.dims == 3 && t <= a.nz - 2 ? a.step : 0.f);
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        p1_t[0][e] = x2fma(e == 0 ? stp : sxhi1, x2sub(ux[e], u0_t[e]), p0_t[0][e]);
        p1_t[1][e] = x2fma(syhi, x2sub(uy[e], u0_t[e]), p0_t[1][e]);
        p1_t[2][e] = x2fma(szhi, x2sub(u0_n[e], u0_t[e]), p0_t[2][e]);
        project2(p1_t[0][e], p1_t[1][e], p1_t[2][e]);
      }
      XP1[t & 1][w][lane] = pack4(p1_t[1][0], p1_t[1][1]);
    }
    if (!__syncthreads_and(ok)) { ring_abort(ring, a, waited, issued); return; }
    waited = q;
    // (c) u^1(t)
    float2 qo[3][2] = {{zero, zero}, {zero, zero}, {zero, zero}};   // p^2(t-1)
    if (t >= zc0 - L) {
      const float2 pxm[2] = {shfl_up2(p1_t[0][1]), p1_t[0][0]};
      const float4 pym4 = XP1[t & 1][wp][lane];
      const float2 pym[2] = {lo2(pym4), hi2(pym4)};
      const float2 mzlo = splat(a.dims == 3 && t >= 1 ? 1.f : 0.f);
      const float2 mzhi = splat(a.dims == 3 && t <= a.nz - 2 ? -1.f : 0.f);
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        float2 dh = e == 0 ? x2mul(mxlo0, pxm[0]) : pxm[1];
        dh = e == 0 ? x2sub(dh, p1_t[0][0]) : x2fma(mxhi1, p1_t[0][1], dh);
        dh = x2fma(mylo, pym[e], dh);
        dh = x2fma(myhi, p1_t[1][e], dh);
        if (a.dims == 3) {
          dh = x2fma(mzlo, p1_prev[2][e], dh);
          dh = x2fma(mzhi, p1_t[2][e], dh);
        }
        u1_t[e] = x2fma(nmu, dh, v_t[e]);
      }
      XU1[t & 1][w][lane] = pack4(u1_t[0], u1_t[1]);
      // (d) p^2(t-1)
      if (t >= zc0 + 1 - L) {
        const float2 ux[2] = {u1_prev[1], lo2(XU1[(t - 1) & 1][w][ln])};
        const float4 uy4 = XU1[(t - 1) & 1][wn][lane];
        const float2 uy[2] = {lo2(uy4), hi2(uy4)};
        const float2 szhi = splat(a.dims == 3 && t - 1 <= a.nz - 2 ? a.step : 0.f);
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          qo[0][e] = x2fma(e == 0 ? stp : sxhi1, x2sub(ux[e], u1_prev[e]), p1_prev[0][e]);
          qo[1][e] = x2fma(syhi, x2sub(uy[e], u1_prev[e]), p1_prev[1][e]);
          qo[2][e] = x2fma(szhi, x2sub(u1_t[e], u1_prev[e]), p1_prev[2][e]);
          project2(qo[0][e], qo[1][e], qo[2][e]);
        }
        if (FINAL) {
          XP2[(t - 1) & 1][w][lane] = pack4(qo[1][0], qo[1][1]);
        } else if (out_pair) {
          const size_t gidx = (static_cast<size_t>(t - 1) * a.ny + gy) * a.nx + gx0;
          *reinterpret_cast<float4*>(a.pout[0] + gidx) = pack4(qo[0][0], qo[0][1]);
          *reinterpret_cast<float4*>(a.pout[1] + gidx) = pack4(qo[1][0], qo[1][1]);
          if (a.dims == 3) *reinterpret_cast<float4*>(a.pout[2] + gidx) = pack4(qo[2][0], qo[2][1]);
        }
      }
    }
    if constexpr (FINAL) {
      __syncthreads();
      // (e) x(t-1) = soft(v - mu D^H p^2, kappa)
      if (t >= zc0 + 1) {
        const int qf = t - 1;
        const float2 pxm[2] = {shfl_up2(qo[0][1]), qo[0][0]};
        const float4 pym4 = XP2[(t - 1) & 1][wp][lane];
        const float2 pym[2] = {lo2(pym4), hi2(pym4)};
        const float2 mzlo = splat(a.dims == 3 && qf >= 1 ? 1.f : 0.f);
        const float2 mzhi = splat(a.dims == 3 && qf <= a.nz - 2 ? -1.f : 0.f);
        float2 xv[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          float2 dh = e == 0 ? x2mul(mxlo0, pxm[0]) : pxm[1];
          dh = e == 0 ? x2sub(dh, qo[0][0]) : x2fma(mxhi1, qo[0][1], dh);
          dh = x2fma(mylo, pym[e], dh);
          dh = x2fma(myhi, qo[1][e], dh);
          if (a.dims == 3) {
            dh = x2fma(mzlo, p2z_prev[e], dh);
            dh = x2fma(mzhi, qo[2][e], dh);
          }
          xv[e] = soft_rsqrt(x2fma(nmu, dh, v_prev[e]), a.kappa);
        }
        unsigned bits = 0u;     // OCC: any non-zero component (sign bits masked below)
        if (out_pair) {
          const size_t gidx = (static_cast<size_t>(qf) * a.ny + gy) * a.nx + gx0;
          if (FISTA) {
            const float2 xp[2] = {lo2(xp4), hi2(xp4)};
            const float2 yk[2] = {lo2(yk4), hi2(yk4)};
            float2 yo[2];
            float d = 0.f;
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              const float2 dx = csub(xv[e], xp[e]);
              d += (yk[e].x - xv[e].x) * dx.x + (yk[e].y - xv[e].y) * dx.y;
              yo[e] = make_float2(xv[e].x + beta * dx.x, xv[e].y + beta * dx.y);
            }
            two_sum_add(dot_hi, dot_lo, d);
            *reinterpret_cast<float4*>(a.y_out + gidx) = pack4(yo[0], yo[1]);
            if (OCC)
              bits = __float_as_uint(xv[0].x) | __float_as_uint(xv[0].y) |
                     __float_as_uint(xv[1].x) | __float_as_uint(xv[1].y) |
                     __float_as_uint(yo[0].x) | __float_as_uint(yo[0].y) |
                     __float_as_uint(yo[1].x) | __float_as_uint(yo[1].y);
          }
          *reinterpret_cast<float4*>(a.x_out + gidx) = pack4(xv[0], xv[1]);
        }
        // plane occupancy for the next forward (same value from every writer)
        if (OCC && __any_sync(0xffffffffu, (bits & 0x7fffffffu) != 0u) && lane == 0)
          occ_s[qf - zc0] = 1;
      }
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        p2z_prev[e] = qo[2][e];
        v_prev[e] = v_t[e];
      }
    }
    // rotate the per-position state to the next plane
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      u0_t[e] = u0_n[e];
      v_t[e] = v_n[e];
      u1_prev[e] = u1_t[e];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        p0_t[c][e] = p0_n[c][e];
        p1_prev[c][e] = p1_t[c][e];
      }
    }
  }
  if (FISTA) {
    // restart inner product: per thread a compensated FP32 sum over its
    // voxels (no FP64 in the plane loop), FP64 across the block and a
    // fixed-order sum over the CTAs by the last one, which updates t and beta
    const double bs = block_sum(static_cast<double>(dot_hi) + static_cast<double>(dot_lo));
    // (block_sum's barriers also publish occ_s)
    const int nblk = gridDim.x;
    const int bid = blockIdx.x;
    if (OCC) {
      if (tid < zc1 - zc0 && occ_s[tid]) {
        a.occ[zc0 + tid] = 1;
        __threadfence();
      }
      __syncthreads();
    }
    __shared__ bool last;
    if (tid == 0) {
      a.fin_partials[bid] = bs;
      __threadfence();
      last = atomicAdd(a.fin_ticket, 1u) == static_cast<unsigned>(nblk - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double v = 0.0;
    for (int b = tid; b < nblk; b += blockDim.x) v += static_cast<volatile double*>(a.fin_partials)[b];
    const double dot = block_sum(v);
    if (tid == 0) {
      fista_update(a.sc, dot);
      *a.fin_ticket = 0;
    }
    if (OCC) {
      // occ[nz] = 1 when some plane is all zero (the forward then reads the
      // per-plane flags; otherwise it propagates every plane unchecked)
      int empty = 0;
      for (int q = tid; q < a.nz; q += blockDim.x)
        empty |= static_cast<volatile int*>(a.occ)[q] == 0;
      empty = __syncthreads_or(empty);
      if (tid == 0) a.occ[a.nz] = empty;
    }
  }
}

// Coordinates (i, j, k) of a flat voxel index that advances by a fixed grid
// stride: the stride is split into (si, sj, sk) once, so that each step is
// two adds with a carry instead of 64-bit divisions.
struct VoxelWalk {
  size_t idx;
  int i, j, k;
  int si, sj, sk, nx, ny;
  __device__ VoxelWalk(size_t start, size_t stride, int nx_, int ny_) : idx(start), nx(nx_), ny(ny_) {
    i = static_cast<int>(start % nx);
    j = static_cast<int>((start / nx) % ny);
    k = static_cast<int>(start / (static_cast<size_t>(nx) * ny));
    si = static_cast<int>(stride % nx);
    sj = static_cast<int>((stride / nx) % ny);
    sk = static_cast<int>(stride / (static_cast<size_t>(nx) * ny));
  }
  __device__ void advance(size_t stride) {
    idx += stride;
    i += si;
    int c = i >= nx;
    i -= c ? nx : 0;
    j += sj + c;
    c = j >= ny;
    j -= c ? ny : 0;
    k += sk + c;
  }
};

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

template <int MODE>
__global__ void __launch_bounds__(kRedThreads) k_finalize(const __grid_constant__ FinArgs a) {
  const size_t nvox = static_cast<size_t>(a.nx) * a.ny * a.nz;
  const float beta = (MODE == FIN_FISTA) ? static_cast<float>(a.sc->beta) : 0.f;
  float local = 0.f;
  double dsum = 0.0;
  int cnt = 0;
  const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
  for (VoxelWalk p(static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x, stride, a.nx, a.ny);
       p.idx < nvox; p.advance(stride)) {
    const size_t idx = p.idx;
    const float2 x = soft(form_u(a, idx, p.i, p.j, p.k), a.kappa);
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
    fista_update(a.sc, dot);
    a.w.tickets[1] = 0;
  }
}

__global__ void k_restart_fixup(const float2* x, float2* y, size_t nvox, const DevScalars* sc) {
  if (!sc->restart_flag) return;
  for (size_t idx = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; idx < nvox;
       idx += static_cast<size_t>(gridDim.x) * blockDim.x)
    y[idx] = x[idx];
}

// ||x||_1 and TV(x) (isotropic forward differences, Neumann boundary) in one
// pass. Each item is four consecutive voxels of a row (nx is a multiple of
// 8), read as 16-byte vectors together with the row below and the plane
// below; per thread a compensated FP32 sum, FP64 across blocks.
__global__ void __launch_bounds__(kRedThreads) k_objective(const float2* x, int nx, int ny, int nz,
                                                           int dims, double lam_l1, double lam_tv,
                                                           DevScalars* sc, RedWork w, double* f_out) {
  const int nq = nx / 4;
  const size_t nitems = static_cast<size_t>(nq) * ny * nz;
  const size_t sy = nx, sz = static_cast<size_t>(nx) * ny;
  float l1h = 0.f, l1l = 0.f, tvh = 0.f, tvl = 0.f;
  const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
  for (VoxelWalk p(static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x, stride, nq, ny);
       p.idx < nitems; p.advance(stride)) {
    const int i = 4 * p.i, j = p.j, k = p.k;
    const size_t idx = (static_cast<size_t>(k) * ny + j) * nx + i;
    const float4* xv = reinterpret_cast<const float4*>(x + idx);
    const float4 a0 = xv[0], a1 = xv[1];
    const float2 c[5] = {lo2(a0), hi2(a0), lo2(a1), hi2(a1),
                         i + 4 < nx ? x[idx + 4] : make_float2(0.f, 0.f)};
    float2 ry[4], rz[4];
    const bool hy = j <= ny - 2, hz = dims == 3 && k <= nz - 2;
    if (hy) {
      const float4* r = reinterpret_cast<const float4*>(x + idx + sy);
      const float4 b0 = r[0], b1 = r[1];
      ry[0] = lo2(b0); ry[1] = hi2(b0); ry[2] = lo2(b1); ry[3] = hi2(b1);
    }
    if (hz) {
      const float4* r = reinterpret_cast<const float4*>(x + idx + sz);
      const float4 b0 = r[0], b1 = r[1];
      rz[0] = lo2(b0); rz[1] = hi2(b0); rz[2] = lo2(b1); rz[3] = hi2(b1);
    }
    float l1 = 0.f, tv = 0.f;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      l1 += sqrtf(c[e].x * c[e].x + c[e].y * c[e].y);
      float g2 = 0.f;
      if (e < 3 || i + 4 < nx) { const float2 d = csub(c[e + 1], c[e]); g2 += d.x * d.x + d.y * d.y; }
      if (hy) { const float2 d = csub(ry[e], c[e]); g2 += d.x * d.x + d.y * d.y; }
      if (hz) { const float2 d = csub(rz[e], c[e]); g2 += d.x * d.x + d.y * d.y; }
      tv += sqrtf(g2);
    }
    two_sum_add(l1h, l1l, l1);
    two_sum_add(tvh, tvl, tv);
  }
  const double dl1 = static_cast<double>(l1h) + static_cast<double>(l1l);
  const double dtv = static_cast<double>(tvh) + static_cast<double>(tvl);
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
  sc->beta_used = 0.0;
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

int tv2_ctas(int nx, int ny, int nz, bool final, int zchunk, int split_tile, int zchunk2) {
  const int tx = final ? kTv2TxF : kTv2Tx, ty = final ? kTv2TyF : kTv2Ty;
  const int ntiles = ((nx + tx - 1) / tx) * ((ny + ty - 1) / ty);
  const int ka = zchunk2 > 0 ? std::min(std::max(split_tile, 0), ntiles) : ntiles;
  const int cb = zchunk2 > 0 ? (ntiles - ka) * ((nz + zchunk2 - 1) / zchunk2) : 0;
  return ka * ((nz + zchunk - 1) / zchunk) + cb;
}

cudaError_t launch_tv_step(bool first, int nsteps, const TvArgs& a, cudaStream_t s, bool final,
                           bool fgp) {
  if (nsteps == 2 && (a.nx & 1)) return cudaErrorInvalidValue;   // pairs of x positions
  if (final && nsteps != 2) return cudaErrorInvalidValue;
  if (fgp && nsteps != 1) return cudaErrorInvalidValue;
  const int tx = nsteps == 2 ? (final ? kTv2TxF : TX2) : TX;
  const int ty = nsteps == 2 ? (final ? kTv2TyF : kTv2Ty) : TY;
  dim3 grid((a.nx + tx - 1) / tx, (a.ny + ty - 1) / ty, (a.nz + a.zchunk - 1) / a.zchunk);
  if (nsteps == 2) grid = dim3(tv2_ctas(a.nx, a.ny, a.nz, final, a.zchunk, a.split_tile, a.zchunk2));
  const bool fista = a.fin_mode == FIN_FISTA;
  auto kern = nsteps == 2
                  ? (final ? (fista ? (a.occ ? (first ? k_tv_step2<true, true, kFinFistaOcc>
                                                      : k_tv_step2<false, true, kFinFistaOcc>)
                                             : (first ? k_tv_step2<true, true, FIN_FISTA>
                                                      : k_tv_step2<false, true, FIN_FISTA>))
                                    : (first ? k_tv_step2<true, true> : k_tv_step2<false, true>))
                           : (first ? k_tv_step2<true, false> : k_tv_step2<false, false>))
                  : (fgp ? (first ? k_tv_step<true, true> : k_tv_step<false, true>)
                         : (first ? k_tv_step<true> : k_tv_step<false>));
  const int bytes = nsteps == 2 ? (final ? TvLayout2<kTv2WarpsF>::kBytes : TvLayout2<kTv2Warps>::kBytes)
                                : TvLayout1::kBytes;
  const int threads = nsteps == 2 ? 32 * (final ? kTv2WarpsF : kTv2Warps) : kTvThreads;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  kern<<<grid, threads, bytes, s>>>(a);
  return cudaGetLastError();
}


cudaError_t encode_tmap(CUtensorMap* tm, CUtensorMapDataType type, int rank, const void* base,
                        const cuuint64_t* dims, const cuuint64_t* strides, const cuuint32_t* box) {
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
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  CUresult r = encode(tm, type, static_cast<cuuint32_t>(rank), const_cast<void*>(base), dims, strides,
                      box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// 3D tensor map over a complex64 volume viewed as float32 [nz][ny][2 nx], box
// of box_rows rows x 2 box_cols floats x 1 plane, zero fill out of bounds.
cudaError_t make_volume_tmap(CUtensorMap* tm, const void* base, int nx, int ny, int nz,
                             int box_rows, int box_cols) {
  const cuuint64_t dims[3] = {static_cast<cuuint64_t>(2 * nx), static_cast<cuuint64_t>(ny),
                              static_cast<cuuint64_t>(nz)};
  const cuuint64_t strides[2] = {static_cast<cuuint64_t>(8) * nx,
                                 static_cast<cuuint64_t>(8) * nx * ny};
  const cuuint32_t box[3] = {static_cast<cuuint32_t>(2 * box_cols), static_cast<cuuint32_t>(box_rows), 1};
  return encode_tmap(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box);
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

// Self-test of the bounded wait the TV kernels use: one warp waits on an
// mbarrier that nothing arrives on (no copy is ever issued to it), gives up
// after `polls` polls and records it in *flag as the TV kernels record a
// failed wait in their error flag; the kernel then returns normally.
__global__ void k_wait_selftest(int* flag, int polls) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) {
    mbar_init(smem_addr(&bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool ok = mbar_wait(smem_addr(&bar), 0, polls);
  if (!__all_sync(0xffffffffu, ok) && threadIdx.x == 0) *flag = 1;
}

cudaError_t launch_wait_selftest(int* flag, int polls, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(flag, polls);
  return cudaGetLastError();
}

cudaError_t launch_init_scalars(DevScalars* sc, int accelerate, int restart, cudaStream_t s) {
  k_init_scalars<<<1, 1, 0, s>>>(sc, accelerate, restart);
  return cudaGetLastError();
}

}  // namespace rihv
