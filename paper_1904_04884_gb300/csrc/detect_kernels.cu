// Particle detection on a reconstructed volume (Section 2, segmentation
// paragraph: a low intensity threshold relative to the maximum, a minimum
// object volume, and intensity-weighted centroids; Section 3.2 uses 2/256 of
// the maximum and 5 voxels).
//
// The threshold decision is taken on float32 squares with every operation
// rounded separately (no fused multiply-add): |x|^2 = re*re + im*im and
// thr^2 = (rel*rel) * max|x|^2, compared strictly.
//
// Components (26-connectivity) come from a lock-free union-find on the label
// array: every masked voxel starts as its own root, unions link the larger
// root to the smaller with atomicMin, so the final root of a component is its
// smallest linear index. Roots are numbered in index order by a block-count
// scan, which makes the component order deterministic; per-component sums
// (weight, weighted coordinates, count) accumulate in FP64.
//
// The same detection also runs on a volume's per-plane COO form (Section 2
// stores volumes plane by plane as lists of their non-zero elements), where
// the work follows the non-zeros instead of the voxels: the threshold is taken
// over the listed values, the entries above it are compacted into a list of
// linear indices (ascending, because COO entries are stored plane by plane in
// row-major order), and union-find runs over that list, each entry finding
// its 13 preceding neighbours by binary search.
#include <cuda_runtime.h>

#include "rihv_internal.cuh"

namespace rihv {
namespace {

constexpr int kDetThreads = 1024;
constexpr int kUfLimit = 1 << 20;   // bound on union/find retries (never reached in practice)

__device__ __forceinline__ float mag2_rn(float2 c) {
  return __fadd_rn(__fmul_rn(c.x, c.x), __fmul_rn(c.y, c.y));
}

__global__ void k_det_max(const float2* x, size_t nvox, unsigned* maxbits) {
  float m = 0.f;
  for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < nvox;
       i += static_cast<size_t>(gridDim.x) * blockDim.x)
    m = fmaxf(m, mag2_rn(x[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(maxbits, __float_as_uint(m));
}

__global__ void k_det_init(const float2* x, size_t nvox, float rel, const unsigned* maxbits,
                           int* label) {
  const float thr2 = __fmul_rn(__fmul_rn(rel, rel), __uint_as_float(*maxbits));
  for (size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < nvox;
       i += static_cast<size_t>(gridDim.x) * blockDim.x)
    label[i] = (mag2_rn(x[i]) > thr2) ? static_cast<int>(i) : -1;
}

__device__ __forceinline__ int uf_find(int* label, int a, int* err) {
  for (int it = 0; it < kUfLimit; ++it) {
    const int p = __ldcg(label + a);
    if (p == a) return a;
    a = p;
  }
  *err = 1;
  return a;
}

__device__ __forceinline__ void uf_union(int* label, int a, int b, int* err) {
  for (int it = 0; it < kUfLimit; ++it) {
    a = uf_find(label, a, err);
    b = uf_find(label, b, err);
    if (a == b) return;
    if (a < b) {
      const int t = a; a = b; b = t;
    }
    // a > b: link root a under b
    const int old = atomicMin(label + a, b);
    if (old == a) return;
    a = old;
  }
  *err = 1;
}

__global__ void k_det_merge(int* label, int nx, int ny, int nz, int* err) {
  const size_t nvox = static_cast<size_t>(nx) * ny * nz;
  for (size_t idx = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; idx < nvox;
       idx += static_cast<size_t>(gridDim.x) * blockDim.x) {
    if (__ldcg(label + idx) < 0) continue;
    const int i = static_cast<int>(idx % nx);
    const size_t r = idx / nx;
    const int j = static_cast<int>(r % ny);
    const int k = static_cast<int>(r / ny);
    // the 13 neighbours that precede this voxel in linear order
    for (int dk = -1; dk <= 0; ++dk)
      for (int dj = -1; dj <= 1; ++dj)
        for (int di = -1; di <= 1; ++di) {
          if (dk == 0 && (dj > 0 || (dj == 0 && di >= 0))) continue;
          const int kk = k + dk, jj = j + dj, ii = i + di;
          if (kk < 0 || jj < 0 || jj >= ny || ii < 0 || ii >= nx) continue;
          const size_t nb = (static_cast<size_t>(kk) * ny + jj) * nx + ii;
          if (__ldcg(label + nb) < 0) continue;
          uf_union(label, static_cast<int>(idx), static_cast<int>(nb), err);
        }
  }
}

__global__ void k_det_flatten(int* label, size_t nvox, int* err) {
  for (size_t idx = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; idx < nvox;
       idx += static_cast<size_t>(gridDim.x) * blockDim.x) {
    if (label[idx] < 0) continue;
    label[idx] = uf_find(label, static_cast<int>(idx), err);
  }
}

// One block per 1024 voxels: count the roots.
__global__ void __launch_bounds__(kDetThreads) k_det_count(const int* label, size_t nvox,
                                                           unsigned* counts) {
  const size_t idx = static_cast<size_t>(blockIdx.x) * kDetThreads + threadIdx.x;
  const int is_root = (idx < nvox && label[idx] == static_cast<int>(idx)) ? 1 : 0;
  const int n = __syncthreads_count(is_root);
  if (threadIdx.x == 0) counts[blockIdx.x] = static_cast<unsigned>(n);
}

// Exclusive scan of counts[0..nb) in place by a single block; total -> *ncomp.
__global__ void __launch_bounds__(kDetThreads) k_det_scan(unsigned* counts, size_t nb, int* ncomp) {
  __shared__ unsigned warp_tot[32];
  __shared__ unsigned carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (size_t base = 0; base < nb; base += kDetThreads) {
    const size_t i = base + threadIdx.x;
    const unsigned v = (i < nb) ? counts[i] : 0u;
    unsigned incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      unsigned w = warp_tot[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += t;
      }
      warp_tot[lane] = w;   // inclusive over warps
    }
    __syncthreads();
    const unsigned before = (wid > 0 ? warp_tot[wid - 1] : 0u) + carry;
    if (i < nb) counts[i] = before + incl - v;
    __syncthreads();
    if (threadIdx.x == kDetThreads - 1) carry = before + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) *ncomp = static_cast<int>(carry);
}

// Roots get compact ids in index order; the root voxel records itself as the
// component's smallest index.
__global__ void __launch_bounds__(kDetThreads) k_det_assign(const int* label, size_t nvox,
                                                            const unsigned* offsets, int* cid,
                                                            long long* first) {
  __shared__ unsigned warp_cnt[32];
  const size_t idx = static_cast<size_t>(blockIdx.x) * kDetThreads + threadIdx.x;
  const bool is_root = idx < nvox && label[idx] == static_cast<int>(idx);
  const unsigned ballot = __ballot_sync(0xffffffffu, is_root);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) warp_cnt[wid] = __popc(ballot);
  __syncthreads();
  if (wid == 0) {
    unsigned w = warp_cnt[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    warp_cnt[lane] = w;
  }
  __syncthreads();
  if (is_root) {
    const unsigned rank = (wid > 0 ? warp_cnt[wid - 1] : 0u) + __popc(ballot & ((1u << lane) - 1u));
    const unsigned c = offsets[blockIdx.x] + rank;
    cid[idx] = static_cast<int>(c);
    first[c] = static_cast<long long>(idx);
  }
}

__global__ void k_det_accum(const float2* x, const int* label, const int* cid, int nx, int ny,
                            int nz, double* stats) {
  const size_t nvox = static_cast<size_t>(nx) * ny * nz;
  for (size_t idx = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; idx < nvox;
       idx += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int root = label[idx];
    if (root < 0) continue;
    const int c = cid[root];
    const int i = static_cast<int>(idx % nx);
    const size_t r = idx / nx;
    const int j = static_cast<int>(r % ny);
    const int k = static_cast<int>(r / ny);
    const double w = static_cast<double>(sqrtf(mag2_rn(x[idx])));
    double* s = stats + static_cast<size_t>(c) * 5;
    atomicAdd(s + 0, w);
    atomicAdd(s + 1, w * i);
    atomicAdd(s + 2, w * j);
    atomicAdd(s + 3, w * k);
    atomicAdd(s + 4, 1.0);
  }
}

// ---- detection on a per-plane COO form -------------------------------------

__global__ void k_coo_max(const float2* vals, long long nnz, unsigned* maxbits) {
  float m = 0.f;
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < nnz;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    m = fmaxf(m, mag2_rn(vals[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(maxbits, __float_as_uint(m));
}

__device__ __forceinline__ float coo_thr2(float rel, const unsigned* maxbits) {
  return __fmul_rn(__fmul_rn(rel, rel), __uint_as_float(*maxbits));
}

// One block per 1024 entries: how many lie above the threshold.
__global__ void __launch_bounds__(kDetThreads) k_coo_count(const float2* vals, long long nnz,
                                                           float rel, const unsigned* maxbits,
                                                           unsigned* counts) {
  const long long i = static_cast<long long>(blockIdx.x) * kDetThreads + threadIdx.x;
  const int hit = (i < nnz && mag2_rn(vals[i]) > coo_thr2(rel, maxbits)) ? 1 : 0;
  const int n = __syncthreads_count(hit);
  if (threadIdx.x == 0) counts[blockIdx.x] = static_cast<unsigned>(n);
}

// Entries above the threshold, in COO order, as linear voxel indices and
// weights |x|; their union-find parents start as themselves.
__global__ void __launch_bounds__(kDetThreads) k_coo_compact_hits(
    const long long* plane_off, const int* rows, const int* cols, const float2* vals,
    long long nnz, int nx, int ny, int nz, float rel, const unsigned* maxbits,
    const unsigned* offsets, long long* lin, float* wgt, int* label) {
  __shared__ unsigned warp_cnt[32];
  const long long i = static_cast<long long>(blockIdx.x) * kDetThreads + threadIdx.x;
  float m2 = 0.f;
  if (i < nnz) m2 = mag2_rn(vals[i]);
  const bool hit = i < nnz && m2 > coo_thr2(rel, maxbits);
  const unsigned ballot = __ballot_sync(0xffffffffu, hit);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) warp_cnt[wid] = __popc(ballot);
  __syncthreads();
  if (wid == 0) {
    unsigned w = warp_cnt[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    warp_cnt[lane] = w;
  }
  __syncthreads();
  if (!hit) return;
  // plane of entry i: the last k with plane_off[k] <= i
  int lo = 0, hi = nz;   // invariant: plane_off[lo] <= i < plane_off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (plane_off[mid] <= i) lo = mid; else hi = mid;
  }
  const unsigned pos = offsets[blockIdx.x] + (wid > 0 ? warp_cnt[wid - 1] : 0u) +
                       __popc(ballot & ((1u << lane) - 1u));
  lin[pos] = (static_cast<long long>(lo) * ny + rows[i]) * nx + cols[i];
  wgt[pos] = sqrtf(m2);
  label[pos] = static_cast<int>(pos);
}

// Position of `key` in the ascending lin[0, n), or -1.
__device__ __forceinline__ int find_sorted(const long long* lin, int n, long long key) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const long long v = __ldg(lin + mid);
    if (v < key) lo = mid + 1; else hi = mid;
  }
  return (lo < n && __ldg(lin + lo) == key) ? lo : -1;
}

__global__ void k_coo_merge(const long long* lin, int m, int* label, int nx, int ny, int* err) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += gridDim.x * blockDim.x) {
    const long long idx = lin[e];
    const int i = static_cast<int>(idx % nx);
    const long long r = idx / nx;
    const int j = static_cast<int>(r % ny);
    const long long k = r / ny;
    // the 13 neighbours that precede this voxel in linear order, hence in the list
    for (int dk = -1; dk <= 0; ++dk)
      for (int dj = -1; dj <= 1; ++dj)
        for (int di = -1; di <= 1; ++di) {
          if (dk == 0 && (dj > 0 || (dj == 0 && di >= 0))) continue;
          const long long kk = k + dk;
          const int jj = j + dj, ii = i + di;
          if (kk < 0 || jj < 0 || jj >= ny || ii < 0 || ii >= nx) continue;
          const int q = find_sorted(lin, e, (kk * ny + jj) * nx + ii);
          if (q >= 0) uf_union(label, e, q, err);
        }
  }
}

__global__ void k_coo_flatten(int* label, int m, int* err) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += gridDim.x * blockDim.x)
    label[e] = uf_find(label, e, err);
}

// Roots (label[e] == e) get compact ids in list order, which is voxel order;
// the component's smallest voxel index is its root's.
__global__ void __launch_bounds__(kDetThreads) k_coo_assign(const int* label, int m,
                                                            const long long* lin,
                                                            const unsigned* offsets, int* cid,
                                                            long long* first) {
  __shared__ unsigned warp_cnt[32];
  const int e = blockIdx.x * kDetThreads + threadIdx.x;
  const bool is_root = e < m && label[e] == e;
  const unsigned ballot = __ballot_sync(0xffffffffu, is_root);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) warp_cnt[wid] = __popc(ballot);
  __syncthreads();
  if (wid == 0) {
    unsigned w = warp_cnt[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    warp_cnt[lane] = w;
  }
  __syncthreads();
  if (is_root) {
    const unsigned c = offsets[blockIdx.x] + (wid > 0 ? warp_cnt[wid - 1] : 0u) +
                       __popc(ballot & ((1u << lane) - 1u));
    cid[e] = static_cast<int>(c);
    first[c] = lin[e];
  }
}

__global__ void k_coo_accum(const long long* lin, const float* wgt, const int* label,
                            const int* cid, int m, int nx, int ny, double* stats) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += gridDim.x * blockDim.x) {
    const int c = cid[label[e]];
    const long long idx = lin[e];
    const int i = static_cast<int>(idx % nx);
    const long long r = idx / nx;
    const int j = static_cast<int>(r % ny);
    const long long k = r / ny;
    const double w = static_cast<double>(wgt[e]);
    double* s = stats + static_cast<size_t>(c) * 5;
    atomicAdd(s + 0, w);
    atomicAdd(s + 1, w * i);
    atomicAdd(s + 2, w * j);
    atomicAdd(s + 3, w * static_cast<double>(k));
    atomicAdd(s + 4, 1.0);
  }
}

int grid_for(size_t n, int threads) {
  size_t b = (n + threads - 1) / threads;
  return static_cast<int>(b < 152 * 16 ? b : 152 * 16);
}

}  // namespace

cudaError_t detect_label(const float2* x, int nx, int ny, int nz, float rel, DetectWork& w,
                         int* err_dev, int* ncomp_host, cudaStream_t s) {
  const size_t nvox = static_cast<size_t>(nx) * ny * nz;
  cudaError_t e = cudaMemsetAsync(w.maxbits, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  k_det_max<<<grid_for(nvox, 256), 256, 0, s>>>(x, nvox, w.maxbits);
  k_det_init<<<grid_for(nvox, 256), 256, 0, s>>>(x, nvox, rel, w.maxbits, w.label);
  k_det_merge<<<grid_for(nvox, 256), 256, 0, s>>>(w.label, nx, ny, nz, err_dev);
  k_det_flatten<<<grid_for(nvox, 256), 256, 0, s>>>(w.label, nvox, err_dev);
  const size_t nb = (nvox + kDetThreads - 1) / kDetThreads;
  k_det_count<<<static_cast<unsigned>(nb), kDetThreads, 0, s>>>(w.label, nvox, w.block_counts);
  k_det_scan<<<1, kDetThreads, 0, s>>>(w.block_counts, nb, w.ncomp);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  e = cudaMemcpyAsync(ncomp_host, w.ncomp, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

cudaError_t detect_stats(const float2* x, int nx, int ny, int nz, DetectWork& w, int ncomp,
                         cudaStream_t s) {
  const size_t nvox = static_cast<size_t>(nx) * ny * nz;
  const size_t nb = (nvox + kDetThreads - 1) / kDetThreads;
  cudaError_t e = cudaMemsetAsync(w.stats, 0, sizeof(double) * 5 * static_cast<size_t>(ncomp), s);
  if (e != cudaSuccess) return e;
  k_det_assign<<<static_cast<unsigned>(nb), kDetThreads, 0, s>>>(w.label, nvox, w.block_counts,
                                                                 w.cid, w.first);
  k_det_accum<<<grid_for(nvox, 256), 256, 0, s>>>(x, w.label, w.cid, nx, ny, nz, w.stats);
  return cudaGetLastError();
}

cudaError_t detect_coo_hits(const long long* plane_off, const int* rows, const int* cols,
                            const float2* vals, long long nnz, int nx, int ny, int nz, float rel,
                            CooDetectWork& w, int* m_host, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(w.maxbits, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  const size_t nb = static_cast<size_t>((nnz + kDetThreads - 1) / kDetThreads);
  k_coo_max<<<grid_for(static_cast<size_t>(nnz), 256), 256, 0, s>>>(vals, nnz, w.maxbits);
  k_coo_count<<<static_cast<unsigned>(nb), kDetThreads, 0, s>>>(vals, nnz, rel, w.maxbits,
                                                                w.block_counts);
  k_det_scan<<<1, kDetThreads, 0, s>>>(w.block_counts, nb, w.nhits);
  k_coo_compact_hits<<<static_cast<unsigned>(nb), kDetThreads, 0, s>>>(
      plane_off, rows, cols, vals, nnz, nx, ny, nz, rel, w.maxbits, w.block_counts, w.lin, w.wgt,
      w.label);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  e = cudaMemcpyAsync(m_host, w.nhits, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

cudaError_t detect_coo_label(int m, int nx, int ny, CooDetectWork& w, int* err_dev, int* ncomp_host,
                             cudaStream_t s) {
  const size_t nb = (static_cast<size_t>(m) + kDetThreads - 1) / kDetThreads;
  k_coo_merge<<<grid_for(m, 256), 256, 0, s>>>(w.lin, m, w.label, nx, ny, err_dev);
  k_coo_flatten<<<grid_for(m, 256), 256, 0, s>>>(w.label, m, err_dev);
  k_det_count<<<static_cast<unsigned>(nb), kDetThreads, 0, s>>>(w.label, static_cast<size_t>(m),
                                                                w.block_counts);
  k_det_scan<<<1, kDetThreads, 0, s>>>(w.block_counts, nb, w.ncomp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(ncomp_host, w.ncomp, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

cudaError_t detect_coo_stats(int m, int nx, int ny, CooDetectWork& w, int ncomp, double* stats,
                             long long* first, cudaStream_t s) {
  const size_t nb = (static_cast<size_t>(m) + kDetThreads - 1) / kDetThreads;
  cudaError_t e = cudaMemsetAsync(stats, 0, sizeof(double) * 5 * static_cast<size_t>(ncomp), s);
  if (e != cudaSuccess) return e;
  k_coo_assign<<<static_cast<unsigned>(nb), kDetThreads, 0, s>>>(w.label, m, w.lin,
                                                                 w.block_counts, w.cid, first);
  k_coo_accum<<<grid_for(m, 256), 256, 0, s>>>(w.lin, w.wgt, w.label, w.cid, m, nx, ny, stats);
  return cudaGetLastError();
}

}  // namespace rihv
