// Per-plane 2D FFT passes for the angular-spectrum forward model and its
// adjoint (Section 2: every depth plane is propagated forward and back).
//
// Design (GB300): a 2D transform of an n_y x n_x plane is a row pass (length
// n_x transforms along x) and a column pass (length n_y along y). Both passes
// run the same shared-memory Stockham engine on a tile of B independent
// transforms stored interleaved, tile[n * (B + 1) + b], so that lanes of a
// warp that work on the same butterfly index touch consecutive words. Radix
// 2/3/4/8 butterflies run in registers, out of place between two tiles;
// twiddles exp(-2 pi i m / n) come from an FP64-computed table staged in
// shared memory. Two CTAs of 512 threads fit on an SM at n = 1024.
//
// Between the passes, planes live in a strip-major intermediate layout
// [z][n_x / W][n_y][W] (W = kStrip) so that one column strip of one plane is a
// single contiguous block.
//
// The forward column pass generates H_j for its strip on the fly from a
// per-frequency phase table read through L2 (uint32 fractions of a cycle:
// phase of plane j is phi0 + j * phid modulo 2^32, exact integer
// accumulation) and sums over the
// planes of its z-group in registers, so per-plane spectra never reach memory.
// The adjoint column pass starts from the residual spectrum R, forms
// conj(H_j) R in registers for every plane and inverse-transforms it.
#include <cuda_runtime.h>

#include "rihv_internal.cuh"

namespace rihv {
namespace {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 rot_i(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

constexpr float kRsqrt2 = 0.70710678118654752440f;
constexpr float kSin60 = 0.86602540378443864676f;

template <int R, bool INV>
struct Dft;

template <bool INV>
struct Dft<2, INV> {
  __device__ __forceinline__ static void run(float2* a) {
    float2 t = a[0];
    a[0] = cadd(t, a[1]);
    a[1] = csub(t, a[1]);
  }
};

template <bool INV>
struct Dft<4, INV> {
  __device__ __forceinline__ static void run(float2* a) {
    float2 t0 = cadd(a[0], a[2]);
    float2 t1 = csub(a[0], a[2]);
    float2 t2 = cadd(a[1], a[3]);
    float2 t3 = rot_i<INV>(csub(a[1], a[3]));
    a[0] = cadd(t0, t2);
    a[2] = csub(t0, t2);
    a[1] = cadd(t1, t3);
    a[3] = csub(t1, t3);
  }
};

template <bool INV>
struct Dft<8, INV> {
  __device__ __forceinline__ static void run(float2* a) {
    float2 e[4] = {a[0], a[2], a[4], a[6]};
    float2 o[4] = {a[1], a[3], a[5], a[7]};
    Dft<4, INV>::run(e);
    Dft<4, INV>::run(o);
    // o[m] *= W8^m, W8 = exp(-+ i pi / 4)
    float2 o1, o3;
    if (!INV) {
      o1 = make_float2(kRsqrt2 * (o[1].x + o[1].y), kRsqrt2 * (o[1].y - o[1].x));
      o3 = make_float2(kRsqrt2 * (o[3].y - o[3].x), -kRsqrt2 * (o[3].x + o[3].y));
    } else {
      o1 = make_float2(kRsqrt2 * (o[1].x - o[1].y), kRsqrt2 * (o[1].x + o[1].y));
      o3 = make_float2(-kRsqrt2 * (o[3].x + o[3].y), kRsqrt2 * (o[3].x - o[3].y));
    }
    float2 o2 = rot_i<INV>(o[2]);
    a[0] = cadd(e[0], o[0]);
    a[4] = csub(e[0], o[0]);
    a[1] = cadd(e[1], o1);
    a[5] = csub(e[1], o1);
    a[2] = cadd(e[2], o2);
    a[6] = csub(e[2], o2);
    a[3] = cadd(e[3], o3);
    a[7] = csub(e[3], o3);
  }
};

template <bool INV>
struct Dft<3, INV> {
  __device__ __forceinline__ static void run(float2* a) {
    float2 t = cadd(a[1], a[2]);
    float2 m = make_float2(a[0].x - 0.5f * t.x, a[0].y - 0.5f * t.y);
    float2 d = cscale(rot_i<INV>(csub(a[1], a[2])), kSin60);
    a[0] = cadd(a[0], t);
    a[1] = cadd(m, d);
    a[2] = csub(m, d);
  }
};

// One out-of-place Stockham pass of radix R over B interleaved transforms of
// length n (tile[n * (B + 1) + b]). Butterfly i (k = i mod p, p = product of
// the radices of earlier passes) reads x[i + j n/R], multiplies input j by
// w^(j k), w = exp(-+2 pi i/(p R)), transforms, and writes output m to
// position (i - k) R + k + m p. Threads take butterflies in turn, each holding
// only its R values, which keeps the register footprint small.
template <int R, int B, bool INV>
__device__ __forceinline__ void fft_pass(const float2* __restrict__ in, float2* __restrict__ out,
                                         int n, int p, const float2* __restrict__ tw) {
  constexpr int LD = B + 1;
  const int nr = n / R;
  const int nbf = nr * B;
  const int tstride = n / (p * R);
  for (int bf = threadIdx.x; bf < nbf; bf += blockDim.x) {
    const int b = bf % B, i = bf / B;
    float2 v[R];
#pragma unroll
    for (int j = 0; j < R; ++j) v[j] = in[(i + j * nr) * LD + b];
    const int k = i % p;
    if (p > 1) {
#pragma unroll
      for (int j = 1; j < R; ++j) {
        const float2 w = tw[j * k * tstride];
        v[j] = INV ? cmulc(v[j], w) : cmul(v[j], w);
      }
    }
    Dft<R, INV>::run(v);
    const int base = (i - k) * R + k;
#pragma unroll
    for (int m = 0; m < R; ++m) out[(base + m * p) * LD + b] = v[m];
  }
  __syncthreads();
}

// Runs all passes of the plan, ping-ponging between two tiles; returns the
// tile holding the result.
template <int B, bool INV>
__device__ __forceinline__ float2* fft_run(float2* t0, float2* t1, const FftPlan& plan,
                                           const float2* tw) {
  int p = 1;
  for (int s = 0; s < plan.npass; ++s) {
    const int r = plan.radix[s];
    if (r == 8)
      fft_pass<8, B, INV>(t0, t1, plan.n, p, tw);
    else if (r == 4)
      fft_pass<4, B, INV>(t0, t1, plan.n, p, tw);
    else if (r == 2)
      fft_pass<2, B, INV>(t0, t1, plan.n, p, tw);
    else
      fft_pass<3, B, INV>(t0, t1, plan.n, p, tw);
    p *= r;
    float2* t = t0;
    t0 = t1;
    t1 = t;
  }
  return t0;
}

__device__ __forceinline__ void stage_twiddles(float2* dst, const float2* src, int n) {
  for (int m = threadIdx.x; m < n; m += blockDim.x) dst[m] = src[m];
}

// ---------------------------------------------------------------------------
// Row pass: kRowsPerCta rows of one plane; transforms along x.
// grid (ny / kRowsPerCta, nz)
// ---------------------------------------------------------------------------
template <bool INV, int IN, int OUT, int EPI>
__global__ void __launch_bounds__(kFftThreads, 2) k_rows(const __grid_constant__ RowArgs a) {
  constexpr int B = kRowsPerCta;
  constexpr int LD = B + 1;
  constexpr int T = kFftThreads;
  constexpr int W = kStrip;
  extern __shared__ float2 smem[];
  const int n = a.nx;
  float2* tile = smem;
  float2* tile2 = smem + n * LD;
  float2* tw = smem + 2 * n * LD;
  stage_twiddles(tw, a.tw, n);

  const int nstrip = a.nx / W;
  const int total = B * n;
  const int rblocks = a.ny / B;
  const int nitems = rblocks * a.nz;
  __syncthreads();

  for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
    const int r0 = (item % rblocks) * B;
    const size_t z = item / rblocks;

    // Load B rows, transposed into the interleaved tile.
    for (int e = threadIdx.x; e < total; e += T) {
      int rl, col;
      float2 val;
      if (IN == ROW_IN_STRIP) {
        const int s = e / (B * W), w = e - s * (B * W);
        rl = w / W;
        col = s * W + (w - rl * W);
        const float2* src = static_cast<const float2*>(a.src);
        val = src[((z * nstrip + s) * a.ny + r0) * W + w];
      } else {
        rl = e / n;
        col = e - rl * n;
        const size_t gi = (z * a.ny + r0 + rl) * a.nx + col;
        if (IN == ROW_IN_F32)
          val = make_float2(static_cast<const float*>(a.src)[gi], 0.f);
        else
          val = static_cast<const float2*>(a.src)[gi];
      }
      tile[col * LD + rl] = val;
    }
    __syncthreads();

    const float2* res = fft_run<B, INV>(tile, tile2, a.plan, tw);

    for (int e = threadIdx.x; e < total; e += T) {
      if (OUT == ROW_OUT_STRIP) {
        const int s = e / (B * W), w = e - s * (B * W);
        const int rl = w / W;
        const int col = s * W + (w - rl * W);
        a.dst[((z * nstrip + s) * a.ny + r0) * W + w] = cscale(res[col * LD + rl], a.scale);
      } else {
        const int rl = e / n, col = e - rl * n;
        const size_t gi = (z * a.ny + r0 + rl) * a.nx + col;
        const float2 g = res[col * LD + rl];
        if (EPI == ROW_EPI_GRAD) {
          const float2 y = a.y[gi];
          a.dst[gi] = make_float2(y.x - a.scale * g.x, y.y - a.scale * g.y);
        } else {
          a.dst[gi] = cscale(g, a.scale);
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Column pass: one strip of kStrip columns; transforms along y.
// grid (nx / kStrip, groups); group g covers planes [g*zpg, min(nz, (g+1)*zpg))
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 transfer(uint2 ph, float amp, int j) {
  const unsigned phi = ph.x + static_cast<unsigned>(j) * ph.y;   // wraps modulo 1 cycle
  const float half_cycles = static_cast<float>(static_cast<int>(phi)) * 4.656612873077393e-10f;  // 2^-31
  float s, c;
  sincospif(half_cycles, &s, &c);
  return make_float2(amp * c, amp * s);
}

template <int MODE>
__global__ void __launch_bounds__(kFftThreads, 2) k_cols(const __grid_constant__ ColArgs a) {
  constexpr int B = kStrip;
  constexpr int LD = B + 1;
  constexpr int T = kFftThreads;
  constexpr int MAXE = kMaxN * B / T;
  extern __shared__ float2 smem[];
  const int n = a.ny;
  const int elems = n * B;
  float2* tile = smem;
  float2* tile2 = smem + n * LD;
  float2* tw = smem + 2 * n * LD;
  stage_twiddles(tw, a.tw, n);

  const int s = blockIdx.x;
  const int nstrip = a.nx / B;
  const size_t strip_elems = static_cast<size_t>(elems);
  const uint2* ph_g = a.phase + s * strip_elems;
  const float* amp_g = a.amp + s * strip_elems;
  __syncthreads();

  if (MODE == COL_FWD_ZSUM) {
    const int z0 = blockIdx.y * a.z_per_group;
    const int z1 = min(a.nz, z0 + a.z_per_group);
    float2 acc[MAXE];
#pragma unroll
    for (int q = 0; q < MAXE; ++q) acc[q] = make_float2(0.f, 0.f);
    for (int z = z0; z < z1; ++z) {
      const float2* src = a.src + (static_cast<size_t>(z) * nstrip + s) * strip_elems;
      for (int e = threadIdx.x; e < elems; e += T) {
        const int r = e / B;
        tile[r * LD + (e - r * B)] = src[e];
      }
      __syncthreads();
      const float2* res = fft_run<B, false>(tile, tile2, a.plan, tw);
#pragma unroll
      for (int q = 0; q < MAXE; ++q) {
        const int e = threadIdx.x + q * T;
        if (e < elems) {
          const int r = e / B;
          const float2 h = transfer(__ldg(ph_g + e), __ldg(amp_g + e), z);
          acc[q] = cadd(acc[q], cmul(h, res[r * LD + (e - r * B)]));
        }
      }
      __syncthreads();
    }
    float2* dst = a.dst + static_cast<size_t>(blockIdx.y) * a.nx * a.ny;
#pragma unroll
    for (int q = 0; q < MAXE; ++q) {
      const int e = threadIdx.x + q * T;
      if (e < elems) {
        const int r = e / B;
        dst[static_cast<size_t>(r) * a.nx + s * B + (e - r * B)] = acc[q];
      }
    }
  } else if (MODE == COL_ADJ_GEN) {
    const int z0 = blockIdx.y * a.z_per_group;
    const int z1 = min(a.nz, z0 + a.z_per_group);
    float2 rr[MAXE];
#pragma unroll
    for (int q = 0; q < MAXE; ++q) {
      const int e = threadIdx.x + q * T;
      rr[q] = make_float2(0.f, 0.f);
      if (e < elems) {
        const int r = e / B;
        rr[q] = cscale(a.src[static_cast<size_t>(r) * a.nx + s * B + (e - r * B)], a.scale);
      }
    }
    for (int z = z0; z < z1; ++z) {
#pragma unroll
      for (int q = 0; q < MAXE; ++q) {
        const int e = threadIdx.x + q * T;
        if (e < elems) {
          const int r = e / B;
          const float2 h = transfer(__ldg(ph_g + e), __ldg(amp_g + e), z);
          tile[r * LD + (e - r * B)] = cmulc(rr[q], h);
        }
      }
      __syncthreads();
      const float2* res = fft_run<B, true>(tile, tile2, a.plan, tw);
      float2* dst = a.dst + (static_cast<size_t>(z) * nstrip + s) * strip_elems;
      for (int e = threadIdx.x; e < elems; e += T) {
        const int r = e / B;
        dst[e] = res[r * LD + (e - r * B)];
      }
      __syncthreads();
    }
  } else if (MODE == COL_PLAIN_FWD) {
    // strip-major plane 0 -> row-major spectrum
    const float2* src = a.src + static_cast<size_t>(s) * strip_elems;
    for (int e = threadIdx.x; e < elems; e += T) {
      const int r = e / B;
      tile[r * LD + (e - r * B)] = src[e];
    }
    __syncthreads();
    const float2* res = fft_run<B, false>(tile, tile2, a.plan, tw);
    for (int e = threadIdx.x; e < elems; e += T) {
      const int r = e / B;
      a.dst[static_cast<size_t>(r) * a.nx + s * B + (e - r * B)] =
          cscale(res[r * LD + (e - r * B)], a.scale);
    }
  } else {  // COL_PLAIN_INV: row-major spectrum -> strip-major plane 0
    for (int e = threadIdx.x; e < elems; e += T) {
      const int r = e / B;
      tile[r * LD + (e - r * B)] = a.src[static_cast<size_t>(r) * a.nx + s * B + (e - r * B)];
    }
    __syncthreads();
    const float2* res = fft_run<B, true>(tile, tile2, a.plan, tw);
    float2* dst = a.dst + static_cast<size_t>(s) * strip_elems;
    for (int e = threadIdx.x; e < elems; e += T) {
      const int r = e / B;
      dst[e] = cscale(res[r * LD + (e - r * B)], a.scale);
    }
  }
}

// ---------------------------------------------------------------------------
// z-group reduction of the forward spectrum, residual and ||r||^2.
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
  return r;  // valid in thread 0
}

__global__ void __launch_bounds__(kRedThreads) k_zsum(const float2* partial, int groups,
                                                      const float2* bhat, float2* out, int nxy,
                                                      double inv_nxy, DevScalars* sc, RedWork w) {
  double local = 0.0;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nxy; idx += gridDim.x * blockDim.x) {
    float2 acc = partial[idx];
    for (int g = 1; g < groups; ++g) acc = cadd(acc, partial[static_cast<size_t>(g) * nxy + idx]);
    if (bhat) {
      acc = csub(acc, bhat[idx]);
      local += static_cast<double>(acc.x * acc.x + acc.y * acc.y);
    }
    out[idx] = acc;
  }
  if (!bhat) return;
  const double bs = block_sum(local);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    w.partials[blockIdx.x] = bs;
    __threadfence();
    last = atomicAdd(&w.tickets[0], 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double v = 0.0;
  for (int b = threadIdx.x; b < static_cast<int>(gridDim.x); b += blockDim.x)
    v += static_cast<volatile double*>(w.partials)[b];
  const double tot = block_sum(v);
  if (threadIdx.x == 0) {
    const double r2 = tot * inv_nxy;
    sc->rnorm2 = r2;
    if (!isfinite(r2)) sc->nonfinite = 1;
    w.tickets[0] = 0;
  }
}

template <bool INV, int IN, int OUT, int EPI>
cudaError_t launch_rows_t(const RowArgs& a, cudaStream_t s) {
  const size_t smem = rows_smem_bytes(a.nx);
  auto kern = k_rows<INV, IN, OUT, EPI>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  int sms = 152, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int items = (a.ny / kRowsPerCta) * a.nz;
  const int grid = items < 2 * sms ? items : 2 * sms;
  kern<<<grid, kFftThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_cols_t(const ColArgs& a, int groups, cudaStream_t s) {
  const size_t smem = cols_smem_bytes(MODE, a.ny);
  auto kern = k_cols<MODE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  dim3 grid(a.nx / kStrip, groups);
  kern<<<grid, kFftThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

size_t rows_smem_bytes(int nx) {
  return sizeof(float2) * (2 * static_cast<size_t>(nx) * (kRowsPerCta + 1) + nx);
}

size_t cols_smem_bytes(int mode, int ny) {
  (void)mode;
  return sizeof(float2) * (2 * static_cast<size_t>(ny) * (kStrip + 1) + ny);
}

cudaError_t launch_rows(int inv, int in, int out, int epi, const RowArgs& a, cudaStream_t s) {
  if (!inv && in == ROW_IN_C64 && out == ROW_OUT_STRIP && epi == ROW_EPI_SCALE)
    return launch_rows_t<false, ROW_IN_C64, ROW_OUT_STRIP, ROW_EPI_SCALE>(a, s);
  if (!inv && in == ROW_IN_F32 && out == ROW_OUT_STRIP && epi == ROW_EPI_SCALE)
    return launch_rows_t<false, ROW_IN_F32, ROW_OUT_STRIP, ROW_EPI_SCALE>(a, s);
  if (inv && in == ROW_IN_STRIP && out == ROW_OUT_C64 && epi == ROW_EPI_GRAD)
    return launch_rows_t<true, ROW_IN_STRIP, ROW_OUT_C64, ROW_EPI_GRAD>(a, s);
  if (inv && in == ROW_IN_STRIP && out == ROW_OUT_C64 && epi == ROW_EPI_SCALE)
    return launch_rows_t<true, ROW_IN_STRIP, ROW_OUT_C64, ROW_EPI_SCALE>(a, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_cols(int mode, const ColArgs& a, int groups, cudaStream_t s) {
  switch (mode) {
    case COL_FWD_ZSUM: return launch_cols_t<COL_FWD_ZSUM>(a, groups, s);
    case COL_ADJ_GEN: return launch_cols_t<COL_ADJ_GEN>(a, groups, s);
    case COL_PLAIN_FWD: return launch_cols_t<COL_PLAIN_FWD>(a, 1, s);
    case COL_PLAIN_INV: return launch_cols_t<COL_PLAIN_INV>(a, 1, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_zsum(const float2* partial, int groups, const float2* bhat, float2* out,
                        int nx, int ny, DevScalars* sc, RedWork w, cudaStream_t s) {
  const int nxy = nx * ny;
  int blocks = (nxy + kRedThreads - 1) / kRedThreads;
  if (blocks > kRedBlocks) blocks = kRedBlocks;
  k_zsum<<<blocks, kRedThreads, 0, s>>>(partial, groups, bhat, out, nxy, 1.0 / nxy, sc, w);
  return cudaGetLastError();
}

}  // namespace rihv
