// Kernels of the FASTA-style solver (Section 2 solves the problem with a
// forward-backward method after FASTA): the gradient step at a step size the
// host chooses, and the inner products its step-size rule and backtracking
// test need.
//
//   v = x - tau g                                    (k_grad_step)
//   s0 = Re<a - b, c - d>, s1 = ||a - b||^2, s2 = ||c - d||^2   (k_dots)
//
// with complex values read as R^2 (the inner product of R^2n). The sums are
// compensated FP32 per thread (Knuth's TwoSum) and FP64 across threads and
// blocks; the last block to finish (ticket counter) adds the block partials
// in a fixed order, so the result does not depend on scheduling.
#include <cuda_runtime.h>

#include "rihv_internal.cuh"

namespace rihv {
namespace {

__global__ void __launch_bounds__(kRedThreads) k_grad_step(const float2* x, const float2* g,
                                                           float tau, float2* v, size_t n) {
  for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const float2 a = x[i], b = g[i];
    v[i] = make_float2(a.x - tau * b.x, a.y - tau * b.y);
  }
}

__device__ __forceinline__ void add_comp(float& hi, float& lo, float v) {
  const float s = hi + v;
  const float bb = s - hi;
  lo += (hi - (s - bb)) + (v - bb);
  hi = s;
}

__device__ __forceinline__ double block_total(double v) {
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
  return r;   // valid in thread 0
}

// d may be null (taken as 0). Rows 1-3 of the partials, ticket 4.
__global__ void __launch_bounds__(kRedThreads) k_dots(const float2* a, const float2* b,
                                                      const float2* c, const float2* d, size_t n,
                                                      RedWork w, double* out) {
  float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f, h2 = 0.f, l2 = 0.f;
  for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const float2 ai = a[i], bi = b[i], ci = c[i];
    const float2 di = d ? d[i] : make_float2(0.f, 0.f);
    const float ex = ai.x - bi.x, ey = ai.y - bi.y;
    const float fx = ci.x - di.x, fy = ci.y - di.y;
    add_comp(h0, l0, ex * fx + ey * fy);
    add_comp(h1, l1, ex * ex + ey * ey);
    add_comp(h2, l2, fx * fx + fy * fy);
  }
  const double t0 = block_total(static_cast<double>(h0) + l0);
  const double t1 = block_total(static_cast<double>(h1) + l1);
  const double t2 = block_total(static_cast<double>(h2) + l2);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    w.partials[1 * kRedBlocks + blockIdx.x] = t0;
    w.partials[2 * kRedBlocks + blockIdx.x] = t1;
    w.partials[3 * kRedBlocks + blockIdx.x] = t2;
    __threadfence();
    last = atomicAdd(&w.tickets[4], 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int r = 0; r < 3; ++r) {
    double v = 0.0;
    for (int blk = threadIdx.x; blk < static_cast<int>(gridDim.x); blk += blockDim.x)
      v += static_cast<volatile double*>(w.partials)[(1 + r) * kRedBlocks + blk];
    const double tot = block_total(v);
    if (threadIdx.x == 0) out[r] = tot;
  }
  if (threadIdx.x == 0) w.tickets[4] = 0;
}

int grid_of(size_t n) {
  const size_t b = (n + kRedThreads - 1) / kRedThreads;
  return static_cast<int>(b < static_cast<size_t>(kRedBlocks) ? b : kRedBlocks);
}

}  // namespace

cudaError_t launch_grad_step(const float2* x, const float2* g, float tau, float2* v, size_t n,
                             cudaStream_t s) {
  k_grad_step<<<grid_of(n), kRedThreads, 0, s>>>(x, g, tau, v, n);
  return cudaGetLastError();
}

cudaError_t launch_dots(const float2* a, const float2* b, const float2* c, const float2* d,
                        size_t n, RedWork w, double* out, cudaStream_t s) {
  k_dots<<<grid_of(n), kRedThreads, 0, s>>>(a, b, c, d, n, w, out);
  return cudaGetLastError();
}

}  // namespace rihv
