// Warm-start network: C ABI of the layer operations and the small
// element-wise / pooling / optimizer kernels around the tcgen05 convolutions.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/rihv_nn.h"
#include "rihv_internal.cuh"

using namespace rihv;

namespace {

__device__ __forceinline__ float bf(uint16_t u) { return __uint_as_float(static_cast<uint32_t>(u) << 16); }
__device__ __forceinline__ uint16_t to_bf(float f) {
  const __nv_bfloat16 b = __float2bfloat16_rn(f);
  return *reinterpret_cast<const uint16_t*>(&b);
}

int grid_for(size_t n, int threads = 256) {
  const size_t b = (n + threads - 1) / threads;
  return static_cast<int>(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

__global__ void k_relu_grad(const uint16_t* g, const uint16_t* y, uint16_t* out, size_t n) {
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x)
    out[i] = bf(y[i]) > 0.f ? g[i] : static_cast<uint16_t>(0);
}

__global__ void k_avgpool2(const uint16_t* x, uint16_t* y, int d, int h, int w, int c) {
  const int od = d / 2, oh = h / 2, ow = w / 2;
  const size_t total = static_cast<size_t>(od) * oh * ow * c;
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int ch = static_cast<int>(i % c);
    size_t v = i / c;
    const int ox = static_cast<int>(v % ow); v /= ow;
    const int oy = static_cast<int>(v % oh);
    const int oz = static_cast<int>(v / oh);
    float s = 0.f;
    for (int k = 0; k < 8; ++k) {
      const int zz = 2 * oz + (k >> 2), yy = 2 * oy + ((k >> 1) & 1), xx = 2 * ox + (k & 1);
      s += bf(x[((static_cast<size_t>(zz) * h + yy) * w + xx) * c + ch]);
    }
    y[i] = to_bf(0.125f * s);
  }
}

__global__ void k_avgpool2_grad(const uint16_t* gy, uint16_t* gx, int d, int h, int w, int c) {
  const size_t total = static_cast<size_t>(d) * h * w * c;
  const int oh = h / 2, ow = w / 2;
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int ch = static_cast<int>(i % c);
    size_t v = i / c;
    const int x = static_cast<int>(v % w); v /= w;
    const int y = static_cast<int>(v % h);
    const int z = static_cast<int>(v / h);
    gx[i] = to_bf(0.125f * bf(gy[((static_cast<size_t>(z / 2) * oh + y / 2) * ow + x / 2) * c + ch]));
  }
}

__global__ void k_upsample2(const uint16_t* x, uint16_t* y, int d, int h, int w, int c) {
  const int od = 2 * d, oh = 2 * h, ow = 2 * w;
  const size_t total = static_cast<size_t>(od) * oh * ow * c;
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int ch = static_cast<int>(i % c);
    size_t v = i / c;
    const int xx = static_cast<int>(v % ow); v /= ow;
    const int yy = static_cast<int>(v % oh);
    const int zz = static_cast<int>(v / oh);
    y[i] = x[((static_cast<size_t>(zz / 2) * h + yy / 2) * w + xx / 2) * c + ch];
  }
}

__global__ void k_upsample2_grad(const uint16_t* gy, uint16_t* gx, int d, int h, int w, int c) {
  const size_t total = static_cast<size_t>(d) * h * w * c;
  const int oh = 2 * h, ow = 2 * w;
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int ch = static_cast<int>(i % c);
    size_t v = i / c;
    const int x = static_cast<int>(v % w); v /= w;
    const int y = static_cast<int>(v % h);
    const int z = static_cast<int>(v / h);
    float s = 0.f;
    for (int k = 0; k < 8; ++k) {
      const int zz = 2 * z + (k >> 2), yy = 2 * y + ((k >> 1) & 1), xx = 2 * x + (k & 1);
      s += bf(gy[((static_cast<size_t>(zz) * oh + yy) * ow + xx) * c + ch]);
    }
    gx[i] = to_bf(s);
  }
}

// ---- 8-channel (16-byte) vector forms, used when every channel count is a
// multiple of 8 and every pointer 16-byte aligned; per channel they add in
// the same order as the scalar forms above, so the results are identical.
__device__ __forceinline__ void unpack8(uint4 u, float* f) {
  const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    f[2 * i] = __uint_as_float(w[i] << 16);
    f[2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
  }
}
__device__ __forceinline__ uint4 pack8(const float* f) {
  uint32_t w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
    w[i] = static_cast<uint32_t>(to_bf(f[2 * i])) | (static_cast<uint32_t>(to_bf(f[2 * i + 1])) << 16);
  return make_uint4(w[0], w[1], w[2], w[3]);
}

__global__ void k_avgpool2_v8(const uint4* x, uint4* y, int d, int h, int w, int g) {
  const int od = d / 2, oh = h / 2, ow = w / 2;
  const size_t total = static_cast<size_t>(od) * oh * ow * g;
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int cg = static_cast<int>(i % g);
    size_t v = i / g;
    const int ox = static_cast<int>(v % ow); v /= ow;
    const int oy = static_cast<int>(v % oh);
    const int oz = static_cast<int>(v / oh);
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int k = 0; k < 8; ++k) {
      const int zz = 2 * oz + (k >> 2), yy = 2 * oy + ((k >> 1) & 1), xx = 2 * ox + (k & 1);
      float f[8];
      unpack8(x[((static_cast<size_t>(zz) * h + yy) * w + xx) * g + cg], f);
#pragma unroll
      for (int j = 0; j < 8; ++j) s[j] += f[j];
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) s[j] *= 0.125f;
    y[i] = pack8(s);
  }
}

__global__ void k_avgpool2_grad_v8(const uint4* gy, uint4* gx, int d, int h, int w, int g) {
  const size_t total = static_cast<size_t>(d) * h * w * g;
  const int oh = h / 2, ow = w / 2;
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int cg = static_cast<int>(i % g);
    size_t v = i / g;
    const int x = static_cast<int>(v % w); v /= w;
    const int y = static_cast<int>(v % h);
    const int z = static_cast<int>(v / h);
    float f[8];
    unpack8(gy[((static_cast<size_t>(z / 2) * oh + y / 2) * ow + x / 2) * g + cg], f);
#pragma unroll
    for (int j = 0; j < 8; ++j) f[j] *= 0.125f;
    gx[i] = pack8(f);
  }
}

__global__ void k_upsample2_v8(const uint4* x, uint4* y, int d, int h, int w, int g) {
  const int od = 2 * d, oh = 2 * h, ow = 2 * w;
  const size_t total = static_cast<size_t>(od) * oh * ow * g;
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int cg = static_cast<int>(i % g);
    size_t v = i / g;
    const int xx = static_cast<int>(v % ow); v /= ow;
    const int yy = static_cast<int>(v % oh);
    const int zz = static_cast<int>(v / oh);
    y[i] = x[((static_cast<size_t>(zz / 2) * h + yy / 2) * w + xx / 2) * g + cg];
  }
}

__global__ void k_upsample2_grad_v8(const uint4* gy, uint4* gx, int d, int h, int w, int g) {
  const size_t total = static_cast<size_t>(d) * h * w * g;
  const int oh = 2 * h, ow = 2 * w;
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int cg = static_cast<int>(i % g);
    size_t v = i / g;
    const int x = static_cast<int>(v % w); v /= w;
    const int y = static_cast<int>(v % h);
    const int z = static_cast<int>(v / h);
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int k = 0; k < 8; ++k) {
      const int zz = 2 * z + (k >> 2), yy = 2 * y + ((k >> 1) & 1), xx = 2 * x + (k & 1);
      float f[8];
      unpack8(gy[((static_cast<size_t>(zz) * oh + yy) * ow + xx) * g + cg], f);
#pragma unroll
      for (int j = 0; j < 8; ++j) s[j] += f[j];
    }
    gx[i] = pack8(s);
  }
}

__global__ void k_concat_v8(const uint4* a, const uint4* b, uint4* out, size_t voxels, int ga, int gb) {
  const int g = ga + gb;
  const size_t total = voxels * g;
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const size_t v = i / g;
    const int cg = static_cast<int>(i - v * g);
    out[i] = cg < ga ? a[v * ga + cg] : b[v * gb + (cg - ga)];
  }
}

__global__ void k_split_v8(const uint4* gsrc, uint4* ga_out, uint4* gb_out, size_t voxels, int ga, int gb) {
  const int g = ga + gb;
  const size_t total = voxels * g;
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const size_t v = i / g;
    const int cg = static_cast<int>(i - v * g);
    if (cg < ga)
      ga_out[v * ga + cg] = gsrc[i];
    else
      gb_out[v * gb + (cg - ga)] = gsrc[i];
  }
}

__global__ void k_pack_input_v8(const float2* vol, uint4* out, size_t voxels, int g, float scale) {
  const size_t total = voxels * g;
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const size_t v = i / g;
    const int cg = static_cast<int>(i - v * g);
    float f[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (cg == 0) {
      const float2 c = vol[v];
      f[0] = scale * c.x;
      f[1] = scale * c.y;
    }
    out[i] = pack8(f);
  }
}

__global__ void k_add(const uint16_t* a, const uint16_t* b, uint16_t* out, size_t n) {
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x)
    out[i] = to_bf(bf(a[i]) + bf(b[i]));
}

__global__ void k_concat(const uint16_t* a, const uint16_t* b, uint16_t* out, size_t voxels, int ca,
                         int cb) {
  const int c = ca + cb;
  const size_t total = voxels * c;
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const size_t v = i / c;
    const int ch = static_cast<int>(i - v * c);
    out[i] = ch < ca ? a[v * ca + ch] : b[v * cb + (ch - ca)];
  }
}

__global__ void k_split(const uint16_t* g, uint16_t* ga, uint16_t* gb, size_t voxels, int ca, int cb) {
  const int c = ca + cb;
  const size_t total = voxels * c;
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const size_t v = i / c;
    const int ch = static_cast<int>(i - v * c);
    if (ch < ca)
      ga[v * ca + ch] = g[i];
    else
      gb[v * cb + (ch - ca)] = g[i];
  }
}

__global__ void k_pack_input(const float2* vol, uint16_t* out, size_t voxels, int c, float scale) {
  const size_t total = voxels * c;
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const size_t v = i / c;
    const int ch = static_cast<int>(i - v * c);
    float val = 0.f;
    if (ch == 0) val = scale * vol[v].x;
    else if (ch == 1) val = scale * vol[v].y;
    out[i] = to_bf(val);
  }
}

__global__ void k_unpack_output(const float* y, const float2* base, float base_scale, float2* vol,
                                size_t voxels, int c, float scale) {
  for (size_t v = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; v < voxels;
       v += static_cast<size_t>(gridDim.x) * blockDim.x) {
    float2 o = make_float2(scale * y[v * c], scale * y[v * c + 1]);
    if (base) {
      const float2 b = base[v];
      o.x += base_scale * b.x;
      o.y += base_scale * b.y;
    }
    vol[v] = o;
  }
}

// Per-channel sums in FP64 over voxel blocks, then a fixed-order final sum.
__global__ void k_bias_grad_partial(const uint16_t* gy, double* part, size_t voxels, int c) {
  // block b handles voxels [b*chunk, ...) for all channels; thread -> channel lane
  const size_t chunk = (voxels + gridDim.x - 1) / gridDim.x;
  const size_t v0 = blockIdx.x * chunk;
  const size_t v1 = v0 + chunk < voxels ? v0 + chunk : voxels;
  for (int ch = threadIdx.x; ch < c; ch += blockDim.x) {
    float s = 0.f;
    double acc = 0.0;
    int cnt = 0;
    for (size_t v = v0; v < v1; ++v) {
      s += bf(gy[v * c + ch]);
      if (++cnt == 64) { acc += s; s = 0.f; cnt = 0; }
    }
    part[static_cast<size_t>(blockIdx.x) * c + ch] = acc + s;
  }
}
// The same on 16-byte vectors of 8 channels (c % 8 == 0): thread t of a block
// takes channel group t % groups of voxels v0 + t / groups, v0 + t / groups +
// per, ... (per = blockDim / groups voxels in step, so consecutive threads
// read consecutive 16-byte words); FP32 sums flushed to FP64 every 64 voxels,
// then per channel a fixed-order sum over the block's threads of its group.
__global__ void __launch_bounds__(256) k_bias_grad_partial_v8(const uint4* gy, double* part,
                                                              size_t voxels, int groups) {
  __shared__ double red[256][8];
  const size_t chunk = (voxels + gridDim.x - 1) / gridDim.x;
  const size_t v0 = blockIdx.x * chunk;
  const size_t v1 = v0 + chunk < voxels ? v0 + chunk : voxels;
  const int per = blockDim.x / groups;
  const int g = threadIdx.x % groups;
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int cnt = 0;
  if (static_cast<int>(threadIdx.x) < per * groups) {
    for (size_t v = v0 + threadIdx.x / groups; v < v1; v += per) {
      const uint4 q = gy[v * groups + g];
      const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        s[2 * j] += __uint_as_float(w[j] << 16);
        s[2 * j + 1] += __uint_as_float(w[j] & 0xFFFF0000u);
      }
      if (++cnt == 64) {
#pragma unroll
        for (int j = 0; j < 8; ++j) { acc[j] += s[j]; s[j] = 0.f; }
        cnt = 0;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) red[threadIdx.x][j] = acc[j] + s[j];
  __syncthreads();
  const int c = groups * 8;
  for (int ch = threadIdx.x; ch < c; ch += blockDim.x) {
    double t = 0.0;
    for (int k = 0; k < per; ++k) t += red[k * groups + ch / 8][ch % 8];
    part[static_cast<size_t>(blockIdx.x) * c + ch] = t;
  }
}

__global__ void k_bias_grad_final(const double* part, int nblocks, float* gb, int c) {
  for (int ch = threadIdx.x; ch < c; ch += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[static_cast<size_t>(b) * c + ch];
    gb[ch] = static_cast<float>(s);
  }
}

__global__ void k_mse_grad(const float* y, const float2* target, uint16_t* gy, double* part,
                           size_t voxels, int c, float inv_scale, float gscale) {
  double local = 0.0;
  for (size_t v = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; v < voxels;
       v += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const float2 t = target[v];
    const float d0 = y[v * c] - inv_scale * t.x;
    const float d1 = y[v * c + 1] - inv_scale * t.y;
    local += static_cast<double>(d0 * d0 + d1 * d1);
    gy[v * c] = to_bf(gscale * d0);
    gy[v * c + 1] = to_bf(gscale * d1);
    for (int ch = 2; ch < c; ++ch) gy[v * c + ch] = 0;
  }
  __shared__ double red[256];
  red[threadIdx.x] = local;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}
__global__ void k_mse_final(const double* part, int nblocks, double* loss, double inv_n) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[b];
    *loss = s * inv_n;
  }
}

__global__ void k_adam(float* p, const float* g, float* m, float* v, uint16_t* pb, size_t n, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    pb[i] = to_bf(pi);
  }
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

rihv_status launched() { return cudaGetLastError() == cudaSuccess ? RIHV_OK : RIHV_ERR_CUDA; }

int device_sms() {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

bool conv_channels_ok(int c_in, int c_out) {
  return c_in >= 16 && c_out >= 16 && c_in % 16 == 0 && c_out % 16 == 0 && c_out <= 256 &&
         c_in <= 256;
}

}  // namespace

extern "C" {

rihv_status rihv_nn_conv3d(const uint16_t* x, const uint16_t* w, const float* bias, void* y, int d,
                           int h, int wd, int c_in, int c_out, int relu, int out_f32, int* err_flag,
                           void* stream) {
  if (!x || !w || !y || !err_flag || d < 1 || h < 1 || wd < 1 || !conv_channels_ok(c_in, c_out) ||
      !aligned16(x) || !aligned16(w) || !aligned16(y))
    return RIHV_ERR_INVALID_ARG;
  ConvArgs a{};
  a.x = reinterpret_cast<const __nv_bfloat16*>(x);
  a.w_ = reinterpret_cast<const __nv_bfloat16*>(w);
  a.bias = bias;
  a.y = y;
  a.d = d;
  a.h = h;
  a.w = wd;
  a.ck = c_in;
  a.n = c_out;
  a.relu = relu;
  a.out_f32 = out_f32;
  a.err = err_flag;
  return launch_conv(false, a, static_cast<cudaStream_t>(stream)) == cudaSuccess ? RIHV_OK
                                                                                 : RIHV_ERR_CUDA;
}

rihv_status rihv_nn_conv3d_dgrad(const uint16_t* gy, const uint16_t* w, void* gx, int d, int h,
                                 int wd, int c_in, int c_out, int out_f32, int* err_flag,
                                 void* stream) {
  if (!gy || !w || !gx || !err_flag || d < 1 || h < 1 || wd < 1 || !conv_channels_ok(c_in, c_out) ||
      !aligned16(gy) || !aligned16(gx))
    return RIHV_ERR_INVALID_ARG;
  ConvArgs a{};
  a.x = reinterpret_cast<const __nv_bfloat16*>(gy);
  a.w_ = reinterpret_cast<const __nv_bfloat16*>(w);
  a.y = gx;
  a.d = d;
  a.h = h;
  a.w = wd;
  a.ck = c_out;
  a.n = c_in;
  a.out_f32 = out_f32;
  a.err = err_flag;
  return launch_conv(true, a, static_cast<cudaStream_t>(stream)) == cudaSuccess ? RIHV_OK
                                                                                : RIHV_ERR_CUDA;
}

size_t rihv_nn_conv3d_wgrad_workspace(int d, int h, int wd, int c_in, int c_out) {
  if (d < 1 || h < 1 || wd < 1 || c_in < 16 || c_out < 16) return 0;
  int ns = 0, tps = 0;
  wgrad_plan(d, h, wd, c_in, device_sms(), &ns, &tps);
  return static_cast<size_t>(ns) * c_out * 27 * c_in * sizeof(float);
}

rihv_status rihv_nn_conv3d_wgrad(const uint16_t* x, const uint16_t* gy, float* gw, int d, int h,
                                 int wd, int c_in, int c_out, void* workspace,
                                 size_t workspace_bytes, int* err_flag, void* stream) {
  if (!x || !gy || !gw || !workspace || !err_flag || d < 1 || h < 1 || wd < 1 ||
      !conv_channels_ok(c_in, c_out) || c_out > 64 || !aligned16(x) || !aligned16(gy) ||
      !aligned16(workspace))
    return RIHV_ERR_INVALID_ARG;
  if (workspace_bytes < rihv_nn_conv3d_wgrad_workspace(d, h, wd, c_in, c_out))
    return RIHV_ERR_INVALID_ARG;
  WgradArgs a{};
  a.x = reinterpret_cast<const __nv_bfloat16*>(x);
  a.gy = reinterpret_cast<const __nv_bfloat16*>(gy);
  a.partial = static_cast<float*>(workspace);
  a.d = d;
  a.h = h;
  a.w = wd;
  a.cin = c_in;
  a.cout = c_out;
  a.err = err_flag;
  wgrad_plan(d, h, wd, c_in, device_sms(), &a.nsplit, &a.tiles_per_split);
  return launch_wgrad(a, gw, static_cast<cudaStream_t>(stream)) == cudaSuccess ? RIHV_OK
                                                                              : RIHV_ERR_CUDA;
}

rihv_status rihv_nn_bias_grad(const uint16_t* gy, float* gb, size_t voxels, int c, void* work,
                              void* stream) {
  if (!gy || !gb || !work || c < 1 || c > 1024 || voxels == 0) return RIHV_ERR_INVALID_ARG;
  const int nb = 256;
  double* part = static_cast<double*>(work);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (c % 8 == 0 && c / 8 <= 256 && aligned16(gy)) {
    const int groups = c / 8;
    const int threads = (256 / groups) * groups;   // a whole number of voxels per step
    k_bias_grad_partial_v8<<<nb, threads, 0, s>>>(reinterpret_cast<const uint4*>(gy), part, voxels,
                                                  groups);
  } else {
    k_bias_grad_partial<<<nb, 128, 0, s>>>(gy, part, voxels, c);
  }
  k_bias_grad_final<<<1, 128, 0, s>>>(part, nb, gb, c);
  return launched();
}

rihv_status rihv_nn_relu_grad(const uint16_t* g, const uint16_t* y, uint16_t* out, size_t n,
                              void* stream) {
  if (!g || !y || !out) return RIHV_ERR_INVALID_ARG;
  k_relu_grad<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(g, y, out, n);
  return launched();
}

rihv_status rihv_nn_avgpool2(const uint16_t* x, uint16_t* y, int d, int h, int wd, int c,
                             void* stream) {
  if (!x || !y || d < 2 || h < 2 || wd < 2 || (d | h | wd) & 1 || c < 1) return RIHV_ERR_INVALID_ARG;
  const size_t n = static_cast<size_t>(d / 2) * (h / 2) * (wd / 2) * c;
  if (c % 8 == 0 && aligned16(x) && aligned16(y))
    k_avgpool2_v8<<<grid_for(n / 8), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const uint4*>(x), reinterpret_cast<uint4*>(y), d, h, wd, c / 8);
  else
    k_avgpool2<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(x, y, d, h, wd, c);
  return launched();
}

rihv_status rihv_nn_avgpool2_grad(const uint16_t* gy, uint16_t* gx, int d, int h, int wd, int c,
                                  void* stream) {
  if (!gy || !gx || d < 2 || h < 2 || wd < 2 || (d | h | wd) & 1 || c < 1) return RIHV_ERR_INVALID_ARG;
  const size_t n = static_cast<size_t>(d) * h * wd * c;
  if (c % 8 == 0 && aligned16(gy) && aligned16(gx))
    k_avgpool2_grad_v8<<<grid_for(n / 8), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const uint4*>(gy), reinterpret_cast<uint4*>(gx), d, h, wd, c / 8);
  else
    k_avgpool2_grad<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(gy, gx, d, h, wd, c);
  return launched();
}

rihv_status rihv_nn_upsample2(const uint16_t* x, uint16_t* y, int d, int h, int wd, int c,
                              void* stream) {
  if (!x || !y || d < 1 || h < 1 || wd < 1 || c < 1) return RIHV_ERR_INVALID_ARG;
  const size_t n = static_cast<size_t>(8) * d * h * wd * c;
  if (c % 8 == 0 && aligned16(x) && aligned16(y))
    k_upsample2_v8<<<grid_for(n / 8), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const uint4*>(x), reinterpret_cast<uint4*>(y), d, h, wd, c / 8);
  else
    k_upsample2<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(x, y, d, h, wd, c);
  return launched();
}

rihv_status rihv_nn_upsample2_grad(const uint16_t* gy, uint16_t* gx, int d, int h, int wd, int c,
                                   void* stream) {
  if (!gy || !gx || d < 1 || h < 1 || wd < 1 || c < 1) return RIHV_ERR_INVALID_ARG;
  const size_t n = static_cast<size_t>(d) * h * wd * c;
  if (c % 8 == 0 && aligned16(gy) && aligned16(gx))
    k_upsample2_grad_v8<<<grid_for(n / 8), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const uint4*>(gy), reinterpret_cast<uint4*>(gx), d, h, wd, c / 8);
  else
    k_upsample2_grad<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(gy, gx, d, h, wd, c);
  return launched();
}

rihv_status rihv_nn_add(const uint16_t* a, const uint16_t* b, uint16_t* out, size_t n,
                        void* stream) {
  if (!a || !b || !out) return RIHV_ERR_INVALID_ARG;
  k_add<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(a, b, out, n);
  return launched();
}

rihv_status rihv_nn_concat(const uint16_t* a, const uint16_t* b, uint16_t* out, size_t voxels,
                           int ca, int cb, void* stream) {
  if (!a || !b || !out || ca < 1 || cb < 1) return RIHV_ERR_INVALID_ARG;
  if (ca % 8 == 0 && cb % 8 == 0 && aligned16(a) && aligned16(b) && aligned16(out))
    k_concat_v8<<<grid_for(voxels * (ca + cb) / 8), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const uint4*>(a), reinterpret_cast<const uint4*>(b), reinterpret_cast<uint4*>(out),
        voxels, ca / 8, cb / 8);
  else
    k_concat<<<grid_for(voxels * (ca + cb)), 256, 0, static_cast<cudaStream_t>(stream)>>>(a, b, out, voxels,
                                                                                       ca, cb);
  return launched();
}

rihv_status rihv_nn_split(const uint16_t* g, uint16_t* ga, uint16_t* gb, size_t voxels, int ca,
                          int cb, void* stream) {
  if (!g || !ga || !gb || ca < 1 || cb < 1) return RIHV_ERR_INVALID_ARG;
  if (ca % 8 == 0 && cb % 8 == 0 && aligned16(g) && aligned16(ga) && aligned16(gb))
    k_split_v8<<<grid_for(voxels * (ca + cb) / 8), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const uint4*>(g), reinterpret_cast<uint4*>(ga), reinterpret_cast<uint4*>(gb),
        voxels, ca / 8, cb / 8);
  else
    k_split<<<grid_for(voxels * (ca + cb)), 256, 0, static_cast<cudaStream_t>(stream)>>>(g, ga, gb, voxels,
                                                                                      ca, cb);
  return launched();
}

rihv_status rihv_nn_pack_input(const void* vol, uint16_t* out, size_t voxels, int c, float scale,
                               void* stream) {
  if (!vol || !out || c < 2) return RIHV_ERR_INVALID_ARG;
  if (c % 8 == 0 && aligned16(out))
    k_pack_input_v8<<<grid_for(voxels * c / 8), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const float2*>(vol), reinterpret_cast<uint4*>(out), voxels, c / 8, scale);
  else
    k_pack_input<<<grid_for(voxels * c), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const float2*>(vol), out, voxels, c, scale);
  return launched();
}

rihv_status rihv_nn_unpack_output(const float* y, const void* base, float base_scale, void* vol,
                                  size_t voxels, int c, float scale, void* stream) {
  if (!y || !vol || c < 2) return RIHV_ERR_INVALID_ARG;
  k_unpack_output<<<grid_for(voxels), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      y, static_cast<const float2*>(base), base_scale, static_cast<float2*>(vol), voxels, c, scale);
  return launched();
}

rihv_status rihv_nn_mse_grad(const float* y, const void* target, uint16_t* gy, double* loss,
                             size_t voxels, int c, float scale, void* work, void* stream) {
  if (!y || !target || !gy || !loss || !work || c < 2 || voxels == 0 || !(scale > 0.f))
    return RIHV_ERR_INVALID_ARG;
  const int nb = 1024;
  double* part = static_cast<double*>(work);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  k_mse_grad<<<nb, 256, 0, s>>>(y, static_cast<const float2*>(target), gy, part, voxels, c,
                                1.f / scale, static_cast<float>(2.0 / static_cast<double>(voxels)));
  k_mse_final<<<1, 32, 0, s>>>(part, nb, loss, 1.0 / static_cast<double>(voxels));
  return launched();
}

rihv_status rihv_nn_adam(float* p, const float* g, float* m, float* v, uint16_t* pb, size_t n,
                         float lr, float b1, float b2, float eps, int step, void* stream) {
  if (!p || !g || !m || !v || !pb || step < 1) return RIHV_ERR_INVALID_ARG;
  const float c1 = 1.f - powf(b1, static_cast<float>(step));
  const float c2 = 1.f - powf(b2, static_cast<float>(step));
  k_adam<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(p, g, m, v, pb, n, lr, b1, b2,
                                                                     eps, c1, c2);
  return launched();
}

}  // extern "C"
