// 3x3x3 convolutions of the warm-start network on 5th-generation tensor cores
// (tcgen05, BF16 operands, FP32 accumulators in tensor memory).
//
// Activations are channels-last, [voxel][channel] in BF16, voxel = (z*H + y)*W + x.
// Weights are W[c_out][tap][c_in], tap = (dz+1)*9 + (dy+1)*3 + (dx+1).
//
// Forward and input gradient (implicit GEMM over a halo tile):
//   D[m][n] = sum_tap sum_k A_tap[m][k] B_tap[n][k]
//   forward : A = X[v_m + off_tap][k],  B = W[n][tap][k]            (n = c_out)
//   dgrad   : A = dY[v_m + off_tap][k], B = W[k][26 - tap][n]       (n = c_in)
// A CTA owns 128 x 2 output voxels (x, y) of one plane. Per 16 input
// channels, TMA brings the 3 x 4 x 130 halo of the tile into shared memory in
// the canonical K-major no-swizzle layout (8 x 16-byte core matrices), so the
// A operand of every tap is a descriptor offset into the same halo; weights
// are staged 9 taps at a time, double buffered; one thread issues the
// tcgen05.mma (M = 128, N = c_out, K = 16) into two TMEM accumulators and
// commits each stage to an mbarrier. The epilogue reads TMEM with tcgen05.ld
// (warp w owns lanes 32w..32w+31), adds the bias, applies ReLU and stores
// BF16 or FP32.
//
// Weight gradient (K = voxels, on the same halo tiles):
//   D_tap[o][c] = sum_v dY[v][o] X[v + off_tap][c]
// A CTA owns one 16-channel input chunk and a run of 128 x 2 voxel tiles.
// Per tile, TMA stages the output gradient [o/8][row][x][8] and the input
// halo of the chunk, double buffered. Both operands are MN-major (for a fixed
// voxel the channels are contiguous): A = dY with M = c_out (rows beyond c_out
// read other shared memory; their results are never read), B = the halo with
// N = 16 channels, and the B operand of tap (dz, dy, dx) is again only a
// descriptor offset into the halo. Each tap accumulates in its own 16 TMEM
// columns (27 x 16 = 432 of 512) over all of the CTA's tiles; the epilogue
// writes FP32 partials per CTA that a second kernel sums in a fixed order.
//
// All waits are bounded: on timeout the CTA records an error, waits (bounded)
// for its issued MMAs, releases its tensor memory and exits.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "rihv_internal.cuh"

namespace rihv {
namespace {

constexpr int kM = 128;                // voxels per CTA tile (MMA M)
constexpr int kThreads = 128;
constexpr int kWaitLimit = 1 << 22;

// ---- PTX helpers -----------------------------------------------------------
__device__ __forceinline__ uint32_t saddr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (int i = 0; i < kWaitLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t dst_slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_slot),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor, no swizzle: start address, leading byte
// offset (along K), stride byte offset (along M/N), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((addr >> 4) & 0x3FFFu);
  d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
  d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
  d |= static_cast<uint64_t>(1) << 46;
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B,
// A/B major-ness (0 = K-major, 1 = MN-major), N >> 3, M >> 4.
__host__ __device__ constexpr uint32_t mma_idesc(int m, int n, int a_mn_major, int b_mn_major) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(a_mn_major) << 15) |
         (static_cast<uint32_t>(b_mn_major) << 16) | (static_cast<uint32_t>(n >> 3) << 17) |
         (static_cast<uint32_t>(m >> 4) << 24);
}

__device__ __forceinline__ uint32_t tmem_cols(int n) {
  uint32_t c = 32;
  while (c < static_cast<uint32_t>(n)) c <<= 1;
  return c;
}

__device__ __forceinline__ void tap_offset(int t, int& dz, int& dy, int& dx) {
  dz = t / 9 - 1;
  dy = (t / 3) % 3 - 1;
  dx = t % 3 - 1;
}

// ---------------------------------------------------------------------------
// Forward / input-gradient kernel (halo tiles by TMA)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* tm, int c0, int c1,
                                            int c2, int c3, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<unsigned long long>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}

// One CTA: a 128 (x) x kTH (y) tile of output voxels in one z plane; kTH
// accumulators of M = 128 rows. The input (16 channels at a time) arrives as
// one TMA box per 8-channel group, [dz][dy][x][8 channels] over the tile's
// 3 x (kTH+2) x 130 halo, zero outside the volume (the convolution's zero
// padding). In that layout the A operand of tap (dz, dy, dx) for output row
// mt is already a K-major operand: rows (voxels) 16 bytes apart inside a core
// matrix, SBO = 128 B between groups of 8 voxels, LBO = one channel group's
// box between the two K halves. So every tap is only a descriptor start
// address, and all 27 taps x kTH rows of MMAs run on one staged halo. The
// weights of 9 taps (one dz plane) are staged per stage in the canonical
// layout, double buffered; one thread issues the MMAs and commits each stage.
template <bool DGRAD>
__global__ void __launch_bounds__(kThreads) k_conv_tile(const __grid_constant__ ConvArgs a,
                                                         const __grid_constant__ ConvMaps maps) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int ck = a.ck;                  // channels of the gathered input (K per tap)
  const int n = a.n;                    // output channels (MMA N)
  const int nchunk = ck / 16;
  const uint32_t wstage_bytes = 9u * n * 32u;
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(smem);   // halo, w0, w1
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 32);
  unsigned char* halo = smem + 128;
  unsigned char* wbuf[2] = {halo + kConvHaloBytes, halo + kConvHaloBytes + wstage_bytes};
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t ncols = tmem_cols(kConvTH * n);
  const int x0 = blockIdx.x * kConvTW, y0 = blockIdx.y * kConvTH, z = blockIdx.z;

  if (tid == 0) {
    for (int i = 0; i < 3; ++i) mbar_init(saddr(&bars[i]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(saddr(tmem_slot), ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = mma_idesc(kM, n, 0, 0);
  const uint32_t halo_a = saddr(halo);
  bool ok = true;
  int stage = 0, last_commit = -1;
  int halo_pending = -1;   // chunk whose halo load may still be in flight

  for (int c = 0; c < nchunk && ok; ++c) {
    // the previous chunk's MMAs read the halo: wait for its last commit
    if (last_commit >= 0) {
      const bool w_ok = mbar_wait(saddr(&bars[1 + (last_commit & 1)]), (last_commit >> 1) & 1);
      ok = __syncthreads_and(w_ok) != 0;
      if (!ok) break;
    }
    if (tid == 0) {
      mbar_expect_tx(saddr(&bars[0]), kConvHaloBytes);
      for (int j = 0; j < 2; ++j)
        tma_load_4d(halo_a + j * kConvHaloKu, &maps.m[2 * c + j], 0, x0 - 1, y0 - 1, z - 1,
                    saddr(&bars[0]));
    }
    halo_pending = c;
    for (int dz = 0; dz < 3 && ok; ++dz, ++stage) {
      const int buf = stage & 1;
      if (stage >= 2) {
        const bool w_ok = mbar_wait(saddr(&bars[1 + buf]), ((stage - 2) >> 1) & 1);
        ok = __syncthreads_and(w_ok) != 0;
        if (!ok) break;
      }
      // weights of taps dz*9 .. dz*9+8, channels 16c .. 16c+15:
      // [tap][n/8][2 K halves][8 rows][16 B]
      for (int u = tid; u < 9 * n * 2; u += kThreads) {
        const int tl = u / (2 * n), rem = u - tl * 2 * n, nn = rem >> 1, j = rem & 1;
        const int t = dz * 9 + tl;
        uint4 val;
        if (!DGRAD) {
          val = __ldg(reinterpret_cast<const uint4*>(a.w_ + (static_cast<size_t>(nn) * 27 + t) * ck) +
                      2 * c + j);
        } else {
          // W is [ck = c_out][27][n = c_in]; B[nn][kk] = W[kk][26 - t][nn]
          uint16_t e[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int kk = (2 * c + j) * 8 + q;
            e[q] = reinterpret_cast<const uint16_t*>(a.w_)[(static_cast<size_t>(kk) * 27 + (26 - t)) * n + nn];
          }
          val = make_uint4(e[0] | (static_cast<uint32_t>(e[1]) << 16), e[2] | (static_cast<uint32_t>(e[3]) << 16),
                           e[4] | (static_cast<uint32_t>(e[5]) << 16), e[6] | (static_cast<uint32_t>(e[7]) << 16));
        }
        *reinterpret_cast<uint4*>(wbuf[buf] + tl * n * 32 + ((nn >> 3) * 2 + j) * 128 + (nn & 7) * 16) = val;
      }
      fence_async_smem();
      if (dz == 0) {
        const bool w_ok = mbar_wait(saddr(&bars[0]), c & 1);
        ok = __syncthreads_and(w_ok) != 0;
        if (!ok) break;
        halo_pending = -1;
      } else {
        __syncthreads();
      }
      if (tid == 0) {
        tc_fence_after();
        const uint32_t b0 = saddr(wbuf[buf]);
        for (int tl = 0; tl < 9; ++tl) {
          const int dy = tl / 3, dx = tl - (tl / 3) * 3;
          const uint64_t bdesc = smem_desc(b0 + tl * n * 32, 128, 256);
#pragma unroll
          for (int mt = 0; mt < kConvTH; ++mt) {
            const uint32_t aoff = ((dz * (kConvTH + 2) + mt + dy) * kConvHX + dx) * 16;
            umma_bf16(tmem + mt * n, smem_desc(halo_a + aoff, kConvHaloKu, 128), bdesc, idesc,
                      (c > 0 || dz > 0 || tl > 0) ? 1u : 0u);
          }
        }
        umma_commit(saddr(&bars[1 + buf]));
      }
      last_commit = stage;
    }
  }

  // all MMAs done: the commit after the last stage
  if (last_commit >= 0) {
    const bool w_ok = mbar_wait(saddr(&bars[1 + (last_commit & 1)]), (last_commit >> 1) & 1);
    ok = (__syncthreads_and(w_ok) != 0) && ok;
  }
  if (!ok) {
    if (tid == 0) {
      atomicExch(a.err, 1);
      if (halo_pending >= 0) mbar_wait(saddr(&bars[0]), halo_pending & 1);   // drain (bounded)
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, ncols);
    return;
  }
  tc_fence_after();
  // epilogue: warp w reads TMEM lanes 32w..32w+31 (voxels x0 + tid) of every row
  const int x = x0 + warp * 32 + lane;
  for (int mt = 0; mt < kConvTH; ++mt) {
    const int y = y0 + mt;
    const bool valid = x < a.w && y < a.h;
    const size_t vo = (static_cast<size_t>(z) * a.h + y) * a.w + x;
    for (int c0 = 0; c0 < n; c0 += 8) {
      float acc[8];
      tmem_ld8(tmem + (static_cast<uint32_t>(warp * 32) << 16) + mt * n + c0, acc);
      if (valid) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (a.bias) acc[j] += a.bias[c0 + j];
          if (a.relu) acc[j] = fmaxf(acc[j], 0.f);
        }
        if (a.out_f32) {
          float4* dst = reinterpret_cast<float4*>(static_cast<float*>(a.y) + vo * n + c0);
          dst[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
          dst[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
        } else {
          __nv_bfloat162 p[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) p[j] = __floats2bfloat162_rn(acc[2 * j], acc[2 * j + 1]);
          *reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(a.y) + vo * n + c0) =
              *reinterpret_cast<uint4*>(p);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, ncols);
}

// ---------------------------------------------------------------------------
// Weight-gradient kernel: grid (splits, input-channel chunks of 16)
// ---------------------------------------------------------------------------
constexpr int kWgGyBytes = 8 * kConvTH * kConvTW * 16;      // 8 groups of c_out (<= 64)
constexpr int kWgStage = kWgGyBytes + kConvHaloBytes;       // gy, then the 16-channel halo
constexpr int kWgSmem = 128 + 2 * kWgStage;
// A descriptors span 16 c_out groups (M = 128) from each stage's gy base
static_assert(128 + kWgStage + 16 * (kWgGyBytes / 8) <= kWgSmem, "wgrad A span exceeds smem");
static_assert(kWgStage % 128 == 0 && kWgGyBytes % 128 == 0, "TMA destinations 128-byte aligned");
constexpr int kWgCols = 512;                                // TMEM columns (27 x 16 used)

struct WgradMaps {
  CUtensorMap x[kConvMaxGroups];   // per 8-channel group of the input, halo box
  CUtensorMap gy[8];               // per 8-channel group of the output gradient, tile box
};

__global__ void __launch_bounds__(kThreads) k_conv_wgrad_tile(const __grid_constant__ WgradArgs a,
                                                               const __grid_constant__ WgradMaps maps) {
  extern __shared__ __align__(1024) unsigned char smem[];
  // bars: 0-1 tile loaded (per stage), 2-3 MMAs of the stage done
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(smem);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 64);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int og = a.cout / 8;
  const int chunk = blockIdx.y;                        // input channels 16 chunk ..
  const int tx = (a.w + kConvTW - 1) / kConvTW, ty = (a.h + kConvTH - 1) / kConvTH;
  const long ntiles = static_cast<long>(tx) * ty * a.d;
  const long t0 = static_cast<long>(blockIdx.x) * a.tiles_per_split;
  const long t1 = t0 + a.tiles_per_split < ntiles ? t0 + a.tiles_per_split : ntiles;
  const int n = t1 > t0 ? static_cast<int>(t1 - t0) : 0;
  const uint32_t tx_bytes = static_cast<uint32_t>(og) * (kWgGyBytes / 8) + kConvHaloBytes;

  if (tid == 0) {
    for (int i = 0; i < 4; ++i) mbar_init(saddr(&bars[i]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(saddr(tmem_slot), kWgCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = mma_idesc(kM, 16, 1, 1);
  const uint32_t base = saddr(smem + 128);

  // tile i of this CTA -> (x0, y0, z), loaded into stage s
  auto issue = [&](int i, int st) {
    const long t = t0 + i;
    const int xt = static_cast<int>(t % tx);
    const long r = t / tx;
    const int y0 = static_cast<int>(r % ty) * kConvTH, z = static_cast<int>(r / ty);
    const int x0 = xt * kConvTW;
    const uint32_t sb = base + st * kWgStage;
    const uint32_t bar = saddr(&bars[st]);
    mbar_expect_tx(bar, tx_bytes);
    for (int g = 0; g < og; ++g)
      tma_load_4d(sb + g * (kWgGyBytes / 8), &maps.gy[g], 0, x0, y0, z, bar);
    for (int j = 0; j < 2; ++j)
      tma_load_4d(sb + kWgGyBytes + j * kConvHaloKu, &maps.x[2 * chunk + j], 0, x0 - 1, y0 - 1,
                  z - 1, bar);
  };

  bool ok = true;
  int loaded_wait = -1;    // last tile whose load was waited for
  int issued = -1;         // last tile whose load was issued
  int committed = -1;      // last tile whose MMAs were committed
  if (tid == 0 && n > 0) {
    issue(0, 0);
    issued = 0;
    for (int i = 0; i < n && ok; ++i) {
      const int st = i & 1;
      ok = mbar_wait(saddr(&bars[st]), (i >> 1) & 1);
      if (!ok) break;
      loaded_wait = i;
      tc_fence_after();
      const uint32_t sg = base + st * kWgStage;
      // descriptors differ only in the start address (bits 0-13, in 16-byte
      // units, no carry: shared addresses stay below 256 KB), so each MMA
      // adds an offset to one of two base descriptors
      const uint64_t ad0 = smem_desc(sg, 128, kWgGyBytes / 8);
      const uint64_t bd0 = smem_desc(sg + kWgGyBytes, 128, kConvHaloKu);
      const uint32_t acc0 = i > 0 ? 1u : 0u;
      for (int dz = 0; dz < 3; ++dz)
        for (int dy = 0; dy < 3; ++dy)
          for (int dx = 0; dx < 3; ++dx) {
            const uint32_t dcol = tmem + (dz * 9 + dy * 3 + dx) * 16;
#pragma unroll
            for (int mt = 0; mt < kConvTH; ++mt) {
              const uint64_t brow = bd0 + ((dz * (kConvTH + 2) + mt + dy) * kConvHX + dx);
              const uint64_t arow = ad0 + mt * (kConvTW * 16 / 16);
#pragma unroll
              for (int k = 0; k < kConvTW / 16; ++k)
                umma_bf16(dcol, arow + k * 16, brow + k * 16, idesc, (acc0 | mt | k) ? 1u : 0u);
            }
          }
      umma_commit(saddr(&bars[2 + st]));
      committed = i;
      if (i + 1 < n) {
        // the other stage held tile i - 1: its MMAs must be done before reuse
        if (i >= 1) {
          ok = mbar_wait(saddr(&bars[2 + (st ^ 1)]), ((i - 1) >> 1) & 1);
          if (!ok) break;
        }
        issue(i + 1, st ^ 1);
        issued = i + 1;
      }
    }
    if (ok && committed >= 0) ok = mbar_wait(saddr(&bars[2 + (committed & 1)]), (committed >> 1) & 1);
    if (!ok) {
      atomicExch(a.err, 1);
      // bounded drains: loads in flight, then the last commit
      for (int i = loaded_wait + 1; i <= issued; ++i) mbar_wait(saddr(&bars[i & 1]), (i >> 1) & 1);
      if (committed >= 0) mbar_wait(saddr(&bars[2 + (committed & 1)]), (committed >> 1) & 1);
    }
  }
  tc_fence_before();
  ok = __syncthreads_and(tid != 0 || ok) != 0;
  tc_fence_after();
  if (ok) {
    // warp w reads TMEM lanes 32w..32w+31 (c_out row o); 27 x 16 columns
    const int o = warp * 32 + lane;
    const int cin = a.cin;
    float* dst = a.partial + (static_cast<size_t>(blockIdx.x) * a.cout + o) * 27 * cin + chunk * 16;
    for (int col = 0; col < 27 * 16; col += 8) {
      float acc[8];
      if (n > 0) {
        tmem_ld8(tmem + (static_cast<uint32_t>(warp * 32) << 16) + col, acc);
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j] = 0.f;
      }
      if (o < a.cout) {
        const int t = col / 16, c = col % 16;
        float4* d4 = reinterpret_cast<float4*>(dst + t * cin + c);
        d4[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
        d4[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kWgCols);
}

// gW[i] = sum over splits of partial[split][i], i = (o * 27 + t) * cin + c (fixed order)
__global__ void k_wgrad_reduce(const float* partial, int nsplit, int total, float* gw) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int sp = 0; sp < nsplit; ++sp) s += partial[static_cast<size_t>(sp) * total + i];
    gw[i] = s;
  }
}

}  // namespace

size_t conv_smem_bytes(int ck, int n) {
  (void)ck;
  return 128 + kConvHaloBytes + 2 * 9 * static_cast<size_t>(n) * 32;
}
cudaError_t launch_conv(bool dgrad, const ConvArgs& a, cudaStream_t s) {
  // one 4D tensor map per 8-channel group of the gathered input:
  // dims (8 channels, x, y, z), box (8, 130, kTH + 2, 3), zero fill
  ConvMaps maps;
  const int groups = a.ck / 8;
  if (groups > kConvMaxGroups || a.ck % 16 != 0) return cudaErrorInvalidValue;
  const cuuint64_t dims[4] = {8, static_cast<cuuint64_t>(a.w), static_cast<cuuint64_t>(a.h),
                              static_cast<cuuint64_t>(a.d)};
  const cuuint64_t row = static_cast<cuuint64_t>(a.ck) * 2;
  const cuuint64_t strides[3] = {row, row * a.w, row * a.w * a.h};
  const cuuint32_t box[4] = {8, kConvHX, kConvTH + 2, 3};
  for (int g = 0; g < groups; ++g) {
    cudaError_t e = encode_tmap(&maps.m[g], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, a.x + g * 8, dims,
                                strides, box);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((a.w + kConvTW - 1) / kConvTW, (a.h + kConvTH - 1) / kConvTH, a.d);
  const size_t smem = conv_smem_bytes(a.ck, a.n);
  auto kern = dgrad ? k_conv_tile<true> : k_conv_tile<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  kern<<<grid, kThreads, smem, s>>>(a, maps);
  return cudaGetLastError();
}

void wgrad_plan(int d, int h, int w, int cin, int sms, int* nsplit, int* tiles_per_split) {
  // one CTA per SM over all input-channel chunks (shared memory and TMEM
  // allow one per SM); the tiles split evenly
  const long tiles = static_cast<long>((w + kConvTW - 1) / kConvTW) * ((h + kConvTH - 1) / kConvTH) * d;
  const int chunks = cin / 16;
  long ns = sms / chunks;          // at most one wave
  if (ns > tiles) ns = tiles;
  if (ns < 1) ns = 1;
  *tiles_per_split = static_cast<int>((tiles + ns - 1) / ns);
  *nsplit = static_cast<int>((tiles + *tiles_per_split - 1) / *tiles_per_split);
}

cudaError_t launch_wgrad(const WgradArgs& a, float* gw, cudaStream_t s) {
  if (a.cin % 16 != 0 || a.cin / 8 > kConvMaxGroups || a.cout % 8 != 0 || a.cout > 64)
    return cudaErrorInvalidValue;
  WgradMaps maps;
  const cuuint32_t xbox[4] = {8, kConvHX, kConvTH + 2, 3};
  const cuuint64_t dims[4] = {8, static_cast<cuuint64_t>(a.w), static_cast<cuuint64_t>(a.h),
                              static_cast<cuuint64_t>(a.d)};
  const cuuint64_t xrow = static_cast<cuuint64_t>(a.cin) * 2;
  const cuuint64_t xstr[3] = {xrow, xrow * a.w, xrow * a.w * a.h};
  for (int g = 0; g < a.cin / 8; ++g) {
    cudaError_t e = encode_tmap(&maps.x[g], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, a.x + g * 8, dims,
                                xstr, xbox);
    if (e != cudaSuccess) return e;
  }
  const cuuint32_t gbox[4] = {8, kConvTW, kConvTH, 1};
  const cuuint64_t grow = static_cast<cuuint64_t>(a.cout) * 2;
  const cuuint64_t gstr[3] = {grow, grow * a.w, grow * a.w * a.h};
  for (int g = 0; g < a.cout / 8; ++g) {
    cudaError_t e = encode_tmap(&maps.gy[g], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, a.gy + g * 8, dims,
                                gstr, gbox);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaFuncSetAttribute(k_conv_wgrad_tile, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kWgSmem);
  if (e != cudaSuccess) return e;
  dim3 grid(a.nsplit, a.cin / 16);
  k_conv_wgrad_tile<<<grid, kThreads, kWgSmem, s>>>(a, maps);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int total = a.cout * 27 * a.cin;
  k_wgrad_reduce<<<128, 256, 0, s>>>(a.partial, a.nsplit, total, gw);
  return cudaGetLastError();
}

}  // namespace rihv
