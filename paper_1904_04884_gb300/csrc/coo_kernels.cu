// Per-plane COO compaction and expansion of a complex64 volume (Section 2,
// GPU implementation paragraph: volumes stored plane by plane as the indices
// and values of their non-zero elements).
//
// Compaction is deterministic: plane k's entries appear in row-major order
// (row j, then column i). Three launches: (1) every CTA counts the non-zero
// elements of its 1024-voxel segment of a plane; (2) one CTA turns the
// counts into exclusive segment offsets and per-plane offsets (int64); (3)
// every CTA writes its segment's entries at its offset, ranking them with
// warp ballots in voxel order. Expansion zero-fills the volume and scatters
// the entries, one grid row per plane.
#include <cuda_runtime.h>

#include "rihv_internal.cuh"

namespace rihv {
namespace {

constexpr int kSeg = kCooSeg;              // voxels per segment (one CTA)
constexpr int kThreads = 256;

__device__ __forceinline__ bool nonzero(float2 v) { return v.x != 0.f || v.y != 0.f; }

// grid (segments per plane, nz)
__global__ void __launch_bounds__(kThreads) k_coo_count(const float2* __restrict__ x, int nxy,
                                                         int* __restrict__ counts) {
  const int seg = blockIdx.x, k = blockIdx.y;
  const size_t base = static_cast<size_t>(k) * nxy + static_cast<size_t>(seg) * kSeg;
  const int lim = min(kSeg, nxy - seg * kSeg);
  int c = 0;
  for (int e = threadIdx.x; e < lim; e += kThreads) c += nonzero(x[base + e]) ? 1 : 0;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  __shared__ int red[kThreads / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    counts[static_cast<size_t>(k) * gridDim.x + seg] = t;
  }
}

// One CTA: exclusive scan of n = nz * segs counts into seg_off (int64), the
// plane offsets (nz + 1) and the total.
__global__ void __launch_bounds__(1024) k_coo_scan(const int* __restrict__ counts, int nz, int segs,
                                                    long long* __restrict__ seg_off,
                                                    long long* __restrict__ plane_off) {
  const int n = nz * segs;
  const int per = (n + blockDim.x - 1) / blockDim.x;
  const int a = threadIdx.x * per, b = min(n, a + per);
  long long s = 0;
  for (int e = a; e < b; ++e) s += counts[e];
  __shared__ long long part[1024];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {             // serial over at most 1024 chunk sums
    long long run = 0;
    for (int t = 0; t < static_cast<int>(blockDim.x); ++t) {
      const long long v = part[t];
      part[t] = run;
      run += v;
    }
  }
  __syncthreads();
  long long run = part[threadIdx.x];
  for (int e = a; e < b; ++e) {
    seg_off[e] = run;
    if (e % segs == 0) plane_off[e / segs] = run;
    run += counts[e];
  }
  if (b == n && a < b) plane_off[nz] = run;
  if (n == 0 && threadIdx.x == 0) plane_off[nz] = 0;
}

// grid (segments per plane, nz): writes the segment's entries in voxel order.
__global__ void __launch_bounds__(kThreads) k_coo_write(const float2* __restrict__ x, int nx, int nxy,
                                                         const long long* __restrict__ seg_off,
                                                         int* __restrict__ rows, int* __restrict__ cols,
                                                         float2* __restrict__ vals) {
  const int seg = blockIdx.x, k = blockIdx.y;
  const size_t base = static_cast<size_t>(k) * nxy + static_cast<size_t>(seg) * kSeg;
  const int lim = min(kSeg, nxy - seg * kSeg);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // each warp owns kSeg / 8 consecutive voxels, processed 32 at a time
  constexpr int kWarpSpan = kSeg / (kThreads / 32);
  __shared__ int wcount[kThreads / 32];
  int mine = 0;
  for (int r = 0; r < kWarpSpan; r += 32) {
    const int e = warp * kWarpSpan + r + lane;
    mine += (e < lim && nonzero(x[base + e])) ? 1 : 0;
  }
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_down_sync(0xffffffffu, mine, o);
  if (lane == 0) wcount[warp] = mine;
  __syncthreads();
  long long pos = seg_off[static_cast<size_t>(k) * gridDim.x + seg];
  for (int w = 0; w < warp; ++w) pos += wcount[w];
  for (int r = 0; r < kWarpSpan; r += 32) {
    const int e = warp * kWarpSpan + r + lane;
    float2 v = make_float2(0.f, 0.f);
    const bool nzv = e < lim && nonzero(v = x[base + e]);
    const unsigned m = __ballot_sync(0xffffffffu, nzv);
    if (nzv) {
      const long long at = pos + __popc(m & ((1u << lane) - 1u));
      const int p = seg * kSeg + e;          // in-plane linear index
      rows[at] = p / nx;
      cols[at] = p - (p / nx) * nx;
      vals[at] = v;
    }
    pos += __popc(m);
  }
}

// grid (blocks, nz): scatter plane k's entries into the zeroed volume.
__global__ void __launch_bounds__(kThreads) k_coo_scatter(const int* __restrict__ rows,
                                                           const int* __restrict__ cols,
                                                           const float2* __restrict__ vals,
                                                           const long long* __restrict__ plane_off,
                                                           int nx, int ny, float2* __restrict__ x,
                                                           int* __restrict__ bad) {
  const int k = blockIdx.y;
  const long long a = plane_off[k], b = plane_off[k + 1];
  const size_t pbase = static_cast<size_t>(k) * nx * ny;
  for (long long e = a + blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < b;
       e += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int r = rows[e], c = cols[e];
    if (r < 0 || r >= ny || c < 0 || c >= nx) {   // malformed entry: skip, report
      atomicExch(bad, 1);
      continue;
    }
    x[pbase + static_cast<size_t>(r) * nx + c] = vals[e];
  }
}

}  // namespace

int coo_segments(int nx, int ny) { return (nx * ny + kSeg - 1) / kSeg; }

cudaError_t launch_coo_count(const float2* x, int nx, int ny, int nz, int* counts, long long* seg_off,
                             long long* plane_off, cudaStream_t s) {
  const int segs = coo_segments(nx, ny);
  k_coo_count<<<dim3(segs, nz), kThreads, 0, s>>>(x, nx * ny, counts);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_coo_scan<<<1, 1024, 0, s>>>(counts, nz, segs, seg_off, plane_off);
  return cudaGetLastError();
}

cudaError_t launch_coo_write(const float2* x, int nx, int ny, int nz, const long long* seg_off,
                             int* rows, int* cols, float2* vals, cudaStream_t s) {
  const int segs = coo_segments(nx, ny);
  k_coo_write<<<dim3(segs, nz), kThreads, 0, s>>>(x, nx, nx * ny, seg_off, rows, cols, vals);
  return cudaGetLastError();
}

cudaError_t launch_coo_scatter(const int* rows, const int* cols, const float2* vals,
                               const long long* plane_off, int nx, int ny, int nz, float2* x,
                               int* bad, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(x, 0, sizeof(float2) * static_cast<size_t>(nx) * ny * nz, s);
  if (e != cudaSuccess) return e;
  k_coo_scatter<<<dim3(64, nz), kThreads, 0, s>>>(rows, cols, vals, plane_off, nx, ny, x, bad);
  return cudaGetLastError();
}

}  // namespace rihv
