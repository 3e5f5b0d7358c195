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

#include <type_traits>

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
// H_j at one frequency. The phase is exact modulo one cycle (integer
// accumulation); the angle in [-pi, pi) goes to the hardware sine/cosine
// approximation (absolute error about 5e-7 on this range), well inside the
// operators' 1e-5 relative budget and far cheaper than the accurate routine.
__device__ __forceinline__ float2 phase_rot(uint2 ph, int j) {
  const unsigned phi = ph.x + static_cast<unsigned>(j) * ph.y;   // wraps modulo 1 cycle
  const float half_cycles = static_cast<float>(static_cast<int>(phi)) * 4.656612873077393e-10f;  // 2^-31
  float s, c;
  __sincosf(half_cycles * 3.14159265358979f, &s, &c);
  return make_float2(c, s);
}
// H_j at one frequency: the band mask (exactly 0 or 1) times the rotation.
__device__ __forceinline__ float2 transfer(uint2 ph, float amp, int j) {
  const float2 r = phase_rot(ph, j);
  return make_float2(amp * r.x, amp * r.y);
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
// Register-resident engine for power-of-two lengths N (64 ... 1024).
//
// One transform is held by a team of N/8 threads, thread i owning the eight
// elements x[i + (N/8) e], e = 0..7. Every Stockham pass (radix 8, the last
// one 2 or 4 when N is not a power of 8) reads exactly that set: butterfly
// b = i + (N/8) q of radix R takes x[b + j N/R], i.e. element e = q + j (8/R)
// of the thread. Its outputs go to (b - k) R + k + m p (k = b mod p, p the
// product of the earlier radices); for the last pass that is b + m N/R, the
// same per-thread set again, so the result stays in registers in natural
// order. Passes in between exchange through shared memory (one barrier per
// exchange, two buffers alternating), indexed l ^ ((l >> 3) & 15), with NT
// interleaved teams (thread = NT i + team) whose rows are N + 16/NT elements
// apart: every half-warp's 8-byte accesses of all passes are then
// conflict-free for NT = 1, 2, 4 and 8. Twiddles come from a pass-major table
// (pass s: w^(j k) at [(j - 1) P + k]), where lanes on consecutive k read
// consecutive words. The first pass reads from global memory and the last
// writes to it directly.
// ---------------------------------------------------------------------------
constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n >> 1); }

template <int N, int NT = 4>
struct RShape {
  static constexpr int TT = N / 8;                                  // threads per transform
  static constexpr int NP = ilog2c(N) / 3 + (ilog2c(N) % 3 ? 1 : 0);  // passes
  static constexpr int LDX = N + 16 / NT;                           // exchange row stride
  static constexpr int kTeams = NT;                                 // transforms per CTA
  static constexpr int kThreads = kTeams * TT;
  // row passes: registers capped for at least 24 resident warps (about 85 per
  // thread) when the CTA is small enough for several per SM, each waiting
  // only on its own barriers
  static constexpr int kMinBlocks = kThreads < 768 ? 768 / kThreads : 1;
  __host__ __device__ static constexpr int radix(int s) {
    return s < ilog2c(N) / 3 ? 8 : (1 << (ilog2c(N) % 3));
  }
  static constexpr size_t smem_bytes() {
    return sizeof(float2) * (static_cast<size_t>(N) + 2 * kTeams * static_cast<size_t>(LDX));
  }
};

__device__ __forceinline__ int xswz(int l) { return l ^ ((l >> 3) & 15); }

// xswz((b - k) R + k + m P), k = b mod P: the exchange position of output m of
// butterfly b. From P = 64 up, (b - k) R, m P and k occupy disjoint bits and
// the swizzle only changes k's low four bits, so the position is a
// per-thread base plus a compile-time offset m P (for P = 64, bit 3 of the
// base also follows m's parity). Identical to xswz for every position.
template <int R, int P>
__device__ __forceinline__ int xpos(int b, int k, int m) {
  if constexpr (P >= 128)
    return (b - k) * R + (k ^ ((k >> 3) & 15)) + m * P;
  else if constexpr (P == 64)
    return (b - k) * R + ((k ^ (k >> 3)) ^ ((m & 1) << 3)) + m * P;
  else
    return xswz((b - k) * R + k + m * P);
}

// xswz(i + TT e) for i < TT: with TT a multiple of 16 the swizzle term is
// ((i >> 3) + (TT / 8) e) mod 16 and leaves TT e untouched, so the position is
// a per-thread base (at most four distinct ones) plus the offset TT e.
template <int TT>
__device__ __forceinline__ int xrd(int i, int e) {
  if constexpr (TT >= 16)
    return (i ^ (((i >> 3) + (TT / 8) * e) & 15)) + TT * e;
  else
    return xswz(i + TT * e);
}

// Offset of pass s's twiddles in the pass-major table (passes with P = 1 have
// none); the whole table has fewer than N entries.
template <int N>
__host__ __device__ constexpr int rtw_offset(int s) {
  int off = 0, p = 1;
  for (int t = 0; t < s; ++t) {
    const int r = RShape<N>::radix(t);
    if (p > 1) off += (r - 1) * p;
    p *= r;
  }
  return off;
}

// Builds the pass-major table in shared memory from the length-N table
// exp(-2 pi i m / N): entry (j - 1) P + k of pass s is w^(j k N / (P R)).
template <int N>
__device__ __forceinline__ void stage_rtw(float2* dst, const float2* __restrict__ src) {
  static_assert(rtw_offset<N>(RShape<N>::NP) <= N, "twiddle table exceeds its shared buffer");
  int off = 0, p = 1;
#pragma unroll
  for (int s = 0; s < RShape<N>::NP; ++s) {
    const int r = RShape<N>::radix(s);
    if (p > 1) {
      for (int idx = threadIdx.x; idx < (r - 1) * p; idx += blockDim.x) {
        const int j = idx / p + 1, k = idx - (j - 1) * p;
        dst[off + idx] = src[j * k * (N / (p * r))];
      }
      off += (r - 1) * p;
    }
    p *= r;
  }
}

template <int N, bool INV, int S, int P>
__device__ __forceinline__ void rfft_passes(float2 (&v)[8], int i, float2* xa, float2* xb,
                                            const float2* __restrict__ tw) {
  if constexpr (S < RShape<N>::NP) {
    constexpr int R = RShape<N>::radix(S);
    constexpr int TT = RShape<N>::TT;
    constexpr bool LAST = S == RShape<N>::NP - 1;
    float2* xs = (S & 1) ? xb : xa;
#pragma unroll
    for (int q = 0; q < 8 / R; ++q) {
      const int b = i + q * TT;
      const int k = b & (P - 1);
      float2 u[R];
#pragma unroll
      for (int j = 0; j < R; ++j) u[j] = v[q + j * (8 / R)];
      if constexpr (P > 1) {
#pragma unroll
        for (int j = 1; j < R; ++j) {
          const float2 w = tw[rtw_offset<N>(S) + (j - 1) * P + k];
          u[j] = INV ? cmulc(u[j], w) : cmul(u[j], w);
        }
      }
      Dft<R, INV>::run(u);
#pragma unroll
      for (int m = 0; m < R; ++m) {
        if constexpr (LAST)
          v[q + m * (8 / R)] = u[m];
        else
          xs[xpos<R, P>(b, k, m)] = u[m];
      }
    }
    if constexpr (!LAST) {
      __syncthreads();
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = xs[xrd<TT>(i, e)];
    }
    rfft_passes<N, INV, S + 1, P * R>(v, i, xa, xb, tw);
  }
}

// One transform per team; afterwards the caller's buffers are swapped when
// the number of exchanges is odd, so consecutive transforms keep alternating.
template <int N, bool INV>
__device__ __forceinline__ void rfft(float2 (&v)[8], int i, float2*& xa, float2*& xb,
                                     const float2* __restrict__ tw) {
  rfft_passes<N, INV, 0, 1>(v, i, xa, xb, tw);
  if constexpr ((RShape<N>::NP - 1) % 2 == 1) {
    float2* t = xa;
    xa = xb;
    xb = t;
  }
}

// Row pass, register engine: NT rows of one plane per item (team = row; 4 by
// default, 2 or 8 when the autotuner finds them faster for a grid).
template <bool INV, int IN, int OUT, int EPI, int N, int NT_ = 4>
__global__ void __launch_bounds__(RShape<N, NT_>::kThreads, RShape<N, NT_>::kMinBlocks) k_rows_reg(const __grid_constant__ RowArgs a) {
  using Sh = RShape<N, NT_>;
  constexpr int TT = Sh::TT, W = kStrip, NT = Sh::kTeams;
  extern __shared__ float2 smem[];
  float2* tw = smem;
  stage_rtw<N>(tw, a.tw);
  const int i = threadIdx.x / NT, team = threadIdx.x % NT;
  float2* xa = smem + N + team * Sh::LDX;
  float2* xb = xa + NT * Sh::LDX;
  constexpr int nstrip = N / W;
  const int rblocks = a.ny / NT;
  const int nitems = rblocks * a.nz;
  __syncthreads();
  auto load = [&](int item, float2 (&v)[8]) {
    const int row = (item % rblocks) * NT + team;
    const size_t z = item / rblocks;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int c = i + TT * e;
      if (IN == ROW_IN_STRIP) {
        v[e] = static_cast<const float2*>(a.src)[((z * nstrip + c / W) * a.ny + row) * W + (c % W)];
      } else {
        const size_t gi = (z * a.ny + row) * N + c;
        if (IN == ROW_IN_F32)
          v[e] = make_float2(static_cast<const float*>(a.src)[gi], 0.f);
        else
          v[e] = static_cast<const float2*>(a.src)[gi];
      }
    }
  };
  // Items of planes marked all-zero are skipped (the same for the whole CTA).
  // The flags are read only when some plane is marked; otherwise the plain
  // instance of the loop runs, with no flag reads in it.
  const int* occ = (IN != ROW_IN_STRIP && a.occ && __ldg(a.occ + a.nz) != 0) ? a.occ : nullptr;
  auto run = [&](auto skip) {
    constexpr bool SKIP = decltype(skip)::value;
    auto live = [&](int item) { return !SKIP || __ldg(occ + item / rblocks) != 0; };
    // the next item's loads are issued before this item's transform
    float2 nxt[8];
    if (blockIdx.x < nitems && live(blockIdx.x)) load(blockIdx.x, nxt);
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
      const int row = (item % rblocks) * NT + team;
      const size_t z = item / rblocks;
      const bool here = live(item);
      float2 v[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = nxt[e];
      if (item + gridDim.x < nitems && live(item + gridDim.x)) load(item + gridDim.x, nxt);
      if (!here) continue;
      // the gradient step's y is loaded before the transform, so that its
      // latency overlaps the transform and no store waits on a load
      float2 yv[8];
      if (OUT != ROW_OUT_STRIP && EPI == ROW_EPI_GRAD) {
#pragma unroll
        for (int e = 0; e < 8; ++e) yv[e] = a.y[(z * a.ny + row) * N + i + TT * e];
      }
      rfft<N, INV>(v, i, xa, xb, tw);
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int c = i + TT * e;
        if (OUT == ROW_OUT_STRIP) {
          a.dst[((z * nstrip + c / W) * a.ny + row) * W + (c % W)] = cscale(v[e], a.scale);
        } else {
          const size_t gi = (z * a.ny + row) * N + c;
          if (EPI == ROW_EPI_GRAD) {
            a.dst[gi] = make_float2(yv[e].x - a.scale * v[e].x, yv[e].y - a.scale * v[e].y);
          } else {
            a.dst[gi] = cscale(v[e], a.scale);
          }
        }
      }
    }
  };
  if (occ)
    run(std::true_type{});
  else
    run(std::false_type{});
}

// Column pass, register engine: one strip of kStrip columns (team = column),
// transforms of length N = ny along y; element (y, w) of the strip at y*kStrip + w.
template <int MODE, int N>
__global__ void __launch_bounds__(RShape<N>::kThreads) k_cols_reg(const __grid_constant__ ColArgs a) {
  using Sh = RShape<N>;
  constexpr int TT = Sh::TT, W = kStrip, NT = Sh::kTeams;
  static_assert(NT == W, "one team per strip column");
  extern __shared__ float2 smem[];
  float2* tw = smem;
  stage_rtw<N>(tw, a.tw);
  const int i = threadIdx.x / NT, w = threadIdx.x % NT;
  float2* xa = smem + N + w * Sh::LDX;
  float2* xb = xa + NT * Sh::LDX;
  const int s = blockIdx.x;
  const int nstrip = a.nx / W;
  constexpr size_t strip_elems = static_cast<size_t>(N) * W;
  __syncthreads();

  if (MODE == COL_FWD_ZSUM || MODE == COL_ADJ_GEN) {
    const int z0 = blockIdx.y * a.z_per_group;
    const int z1 = min(a.nz, z0 + a.z_per_group);
    // transfer-function phases of this thread's frequencies; the band mask
    // (exactly 0 or 1, the same for every plane) is applied once, outside the
    // plane loop: to the z-sum in the forward, to R in the adjoint
    uint2 ph[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) ph[e] = __ldg(a.phase + s * strip_elems + (i + TT * e) * W + w);
    if (MODE == COL_FWD_ZSUM) {
      float2 acc[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) acc[e] = make_float2(0.f, 0.f);
      // Planes marked all-zero add nothing and are passed over (CTA-uniform).
      // The flags are read only when some plane is marked; otherwise the
      // plain loop runs.
      const int* occ = (a.occ && __ldg(a.occ + a.nz) != 0) ? a.occ : nullptr;
      float2 nxt[8];   // the next plane's loads are issued before this plane's transform
      if (!occ) {
        if (z0 < z1) {
          const float2* src = a.src + (static_cast<size_t>(z0) * nstrip + s) * strip_elems;
#pragma unroll
          for (int e = 0; e < 8; ++e) nxt[e] = src[(i + TT * e) * W + w];
        }
        for (int z = z0; z < z1; ++z) {
          float2 v[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) v[e] = nxt[e];
          if (z + 1 < z1) {
            const float2* src = a.src + (static_cast<size_t>(z + 1) * nstrip + s) * strip_elems;
#pragma unroll
            for (int e = 0; e < 8; ++e) nxt[e] = src[(i + TT * e) * W + w];
          }
          rfft<N, false>(v, i, xa, xb, tw);
#pragma unroll
          for (int e = 0; e < 8; ++e) acc[e] = cadd(acc[e], cmul(phase_rot(ph[e], z), v[e]));
        }
      } else {
        auto next_live = [&](int z) {
          while (z < z1 && __ldg(occ + z) == 0) ++z;
          return z;
        };
        int z = next_live(z0);
        if (z < z1) {
          const float2* src = a.src + (static_cast<size_t>(z) * nstrip + s) * strip_elems;
#pragma unroll
          for (int e = 0; e < 8; ++e) nxt[e] = src[(i + TT * e) * W + w];
        }
        while (z < z1) {
          float2 v[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) v[e] = nxt[e];
          const int zn = next_live(z + 1);
          if (zn < z1) {
            const float2* src = a.src + (static_cast<size_t>(zn) * nstrip + s) * strip_elems;
#pragma unroll
            for (int e = 0; e < 8; ++e) nxt[e] = src[(i + TT * e) * W + w];
          }
          rfft<N, false>(v, i, xa, xb, tw);
#pragma unroll
          for (int e = 0; e < 8; ++e) acc[e] = cadd(acc[e], cmul(phase_rot(ph[e], z), v[e]));
          z = zn;
        }
      }
      float2* dst = a.dst + static_cast<size_t>(blockIdx.y) * a.nx * a.ny;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const float amp = __ldg(a.amp + s * strip_elems + (i + TT * e) * W + w);
        dst[static_cast<size_t>(i + TT * e) * a.nx + s * W + w] = cscale(acc[e], amp);
      }
    } else {
      float2 rr[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const float amp = __ldg(a.amp + s * strip_elems + (i + TT * e) * W + w);
        rr[e] = cscale(cscale(a.src[static_cast<size_t>(i + TT * e) * a.nx + s * W + w], a.scale), amp);
      }
      for (int z = z0; z < z1; ++z) {
        float2 v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = cmulc(rr[e], phase_rot(ph[e], z));
        rfft<N, true>(v, i, xa, xb, tw);
        float2* dst = a.dst + (static_cast<size_t>(z) * nstrip + s) * strip_elems;
#pragma unroll
        for (int e = 0; e < 8; ++e) dst[(i + TT * e) * W + w] = v[e];
      }
    }
  } else if (MODE == COL_PLAIN_FWD) {
    // strip-major plane 0 -> row-major spectrum
    const float2* src = a.src + static_cast<size_t>(s) * strip_elems;
    float2 v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = src[(i + TT * e) * W + w];
    rfft<N, false>(v, i, xa, xb, tw);
#pragma unroll
    for (int e = 0; e < 8; ++e)
      a.dst[static_cast<size_t>(i + TT * e) * a.nx + s * W + w] = cscale(v[e], a.scale);
  } else {  // COL_PLAIN_INV: row-major spectrum -> strip-major plane 0
    float2 v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = a.src[static_cast<size_t>(i + TT * e) * a.nx + s * W + w];
    rfft<N, true>(v, i, xa, xb, tw);
    float2* dst = a.dst + static_cast<size_t>(s) * strip_elems;
#pragma unroll
    for (int e = 0; e < 8; ++e) dst[(i + TT * e) * W + w] = cscale(v[e], a.scale);
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

// The forward of the iterate x_k, summed over z-groups, feeds both the
// objective (data term of x_k) and the next gradient: the residual spectrum of
// y_{k+1} = x_k + beta (x_k - x_{k-1}) follows by linearity from S(x_k) and
// S(x_{k-1}), so y never needs a forward of its own.
__global__ void __launch_bounds__(kRedThreads) k_zsum_next(const float2* partial, int groups,
                                                           const float2* bhat,
                                                           const float2* sx_prev, float2* sx,
                                                           float2* ry, int nxy, double inv_nxy,
                                                           DevScalars* sc, RedWork w) {
  const float beta = sc->restart_flag ? 0.f : static_cast<float>(sc->beta_used);
  double local = 0.0;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nxy; idx += gridDim.x * blockDim.x) {
    float2 acc = partial[idx];
    for (int g = 1; g < groups; ++g) acc = cadd(acc, partial[static_cast<size_t>(g) * nxy + idx]);
    sx[idx] = acc;
    const float2 b = bhat[idx];
    const float2 r = csub(acc, b);
    local += static_cast<double>(r.x * r.x + r.y * r.y);
    float2 yv = acc;
    if (beta != 0.f) {
      const float2 p = sx_prev[idx];
      yv = make_float2(acc.x + beta * (acc.x - p.x), acc.y + beta * (acc.y - p.y));
    }
    ry[idx] = csub(yv, b);
  }
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

template <bool INV, int IN, int OUT, int EPI, int N, int NT>
cudaError_t launch_rows_reg_t(const RowArgs& a, cudaStream_t s) {
  using Sh = RShape<N, NT>;
  auto kern = k_rows_reg<INV, IN, OUT, EPI, N, NT>;
  const int smem = static_cast<int>(Sh::smem_bytes());
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int sms = 152, dev = 0, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Sh::kThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const int items = (a.ny / Sh::kTeams) * a.nz;
  const int grid = items < per_sm * sms ? items : per_sm * sms;
  kern<<<grid, Sh::kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <bool INV, int IN, int OUT, int EPI, int N>
cudaError_t launch_rows_reg(const RowArgs& a, cudaStream_t s) {
  switch (a.teams) {
    case 1: return launch_rows_reg_t<INV, IN, OUT, EPI, N, 1>(a, s);
    case 2: return launch_rows_reg_t<INV, IN, OUT, EPI, N, 2>(a, s);
    case 8: return launch_rows_reg_t<INV, IN, OUT, EPI, N, 8>(a, s);
    default: return launch_rows_reg_t<INV, IN, OUT, EPI, N, 4>(a, s);
  }
}

template <int MODE, int N>
cudaError_t launch_cols_reg(const ColArgs& a, int groups, cudaStream_t s) {
  using Sh = RShape<N>;
  auto kern = k_cols_reg<MODE, N>;
  const int smem = static_cast<int>(Sh::smem_bytes());
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  dim3 grid(a.nx / kStrip, groups);
  kern<<<grid, Sh::kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <bool INV, int IN, int OUT, int EPI>
cudaError_t launch_rows_t(const RowArgs& a, cudaStream_t s) {
  switch (a.nx) {
    case 64: return launch_rows_reg<INV, IN, OUT, EPI, 64>(a, s);
    case 128: return launch_rows_reg<INV, IN, OUT, EPI, 128>(a, s);
    case 256: return launch_rows_reg<INV, IN, OUT, EPI, 256>(a, s);
    case 512: return launch_rows_reg<INV, IN, OUT, EPI, 512>(a, s);
    case 1024: return launch_rows_reg<INV, IN, OUT, EPI, 1024>(a, s);
    default: break;
  }
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
  switch (a.ny) {
    case 64: return launch_cols_reg<MODE, 64>(a, groups, s);
    case 128: return launch_cols_reg<MODE, 128>(a, groups, s);
    case 256: return launch_cols_reg<MODE, 256>(a, groups, s);
    case 512: return launch_cols_reg<MODE, 512>(a, groups, s);
    case 1024: return launch_cols_reg<MODE, 1024>(a, groups, s);
    default: break;
  }
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

// Lengths served by the register engine.
bool reg_length(int n) { return n >= 64 && n <= 1024 && (n & (n - 1)) == 0; }

size_t rows_smem_bytes(int nx, int teams) {
  if (reg_length(nx))
    return sizeof(float2) * (nx + 2 * static_cast<size_t>(teams) * (nx + 16 / teams));
  return sizeof(float2) * (2 * static_cast<size_t>(nx) * (kRowsPerCta + 1) + nx);
}

size_t cols_smem_bytes(int mode, int ny) {
  (void)mode;
  if (reg_length(ny)) return sizeof(float2) * (ny + 2 * 4 * static_cast<size_t>(ny + 4));
  return sizeof(float2) * (2 * static_cast<size_t>(ny) * (kStrip + 1) + ny);
}

int cols_ctas_per_sm(int ny) {
  int per_sm = 2;
  cudaError_t e = cudaSuccess;
  switch (ny) {
    case 64: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cols_reg<COL_FWD_ZSUM, 64>, RShape<64>::kThreads, RShape<64>::smem_bytes()); break;
    case 128: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cols_reg<COL_FWD_ZSUM, 128>, RShape<128>::kThreads, RShape<128>::smem_bytes()); break;
    case 256: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cols_reg<COL_FWD_ZSUM, 256>, RShape<256>::kThreads, RShape<256>::smem_bytes()); break;
    case 512: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cols_reg<COL_FWD_ZSUM, 512>, RShape<512>::kThreads, RShape<512>::smem_bytes()); break;
    case 1024: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cols_reg<COL_FWD_ZSUM, 1024>, RShape<1024>::kThreads, RShape<1024>::smem_bytes()); break;
    default: break;
  }
  return (e == cudaSuccess && per_sm >= 1) ? per_sm : 1;
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

cudaError_t launch_zsum_next(const float2* partial, int groups, const float2* bhat,
                             const float2* sx_prev, float2* sx, float2* ry, int nx, int ny,
                             DevScalars* sc, RedWork w, cudaStream_t s) {
  const int nxy = nx * ny;
  int blocks = (nxy + kRedThreads - 1) / kRedThreads;
  if (blocks > kRedBlocks) blocks = kRedBlocks;
  k_zsum_next<<<blocks, kRedThreads, 0, s>>>(partial, groups, bhat, sx_prev, sx, ry, nxy,
                                             1.0 / nxy, sc, w);
  return cudaGetLastError();
}

}  // namespace rihv
