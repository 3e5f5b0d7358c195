// Internal declarations shared by the librihv translation units.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/rihv.h"

namespace rihv {

// ---------------------------------------------------------------------------
// Argument checks shared by the entry points (rihv_api.cu)
// ---------------------------------------------------------------------------
constexpr int kNotDevicePtr = -1;   // host, unregistered or invalid pointer
constexpr int kManagedPtr = -2;     // managed memory (reachable from every device)
constexpr int kLegacyStream = -3;   // the NULL stream (the current device's)
// Device that holds p (kNotDevicePtr / kManagedPtr otherwise).
int pointer_device(const void* p);
// Device a stream belongs to (kLegacyStream for NULL, kNotDevicePtr on error).
int stream_device(const void* stream);
// Message returned by rihv_last_error(NULL).
void set_global_error(const char* msg);

// ---------------------------------------------------------------------------
// Sizes and launch shapes
// ---------------------------------------------------------------------------
constexpr int kMaxN = 1024;        // largest supported nx, ny
constexpr int kRowsPerCta = 4;     // transforms per CTA in the row pass
constexpr int kStrip = 4;          // strip width of the intermediate layout
constexpr int kFftThreads = 512;   // threads per FFT CTA
constexpr int kMaxPasses = 8;

constexpr int kTvTx = 32;          // TV tile width (x)
constexpr int kTvTy = 8;           // TV tile height (y)
constexpr int kTvThreads = kTvTx * kTvTy;
constexpr int kTvBoxW = kTvTx + 4;  // TMA box width in complex elements (x from i0-2)
constexpr int kTvBoxH1 = kTvTy + 2; // box height, one step per launch (y from j0-1)
constexpr int kTvStages = 4;        // planes in the shared-memory ring
// Two steps per launch: a 60 x 16 output tile; one warp per row of the 19-row
// halo (y from j0-1), each lane two x positions (x from i0-2); box 64 x 20 from
// (i0-2, j0-2); a 3-stage plane ring; one CTA per SM.
constexpr int kTv2Tx = 60;
constexpr int kTv2Ty = 16;
constexpr int kTv2Warps = kTv2Ty + 3;
constexpr int kTv2Threads = 32 * kTv2Warps;
constexpr int kTv2BoxW = kTv2Tx + 4;
constexpr int kTv2BoxH = kTv2Ty + 4;
constexpr int kTv2Stages = 3;
constexpr int kTvMaxChunk = 256;   // largest z-chunk of a fused-finalize TV launch
// The launch with the fused finalize needs one more halo ring on the low
// sides (D^H of the final dual): a 58 x 11 tile, box 64 x 16 from (i0-4,
// j0-3), 15 warps (fewer threads leave room for its extra per-thread state).
constexpr int kTv2TxF = 58;
constexpr int kTv2TyF = 11;
constexpr int kTv2WarpsF = kTv2TyF + 4;
constexpr int kTv2BoxHF = kTv2WarpsF + 1;

constexpr int kRedBlocks = 1216;   // fixed grid of the streaming reduction kernels (8 x 152)
constexpr int kRedThreads = 256;

// Radix plan of one 1D transform of length n = product of radix[0..npass).
struct FftPlan {
  int n;
  int npass;
  int radix[kMaxPasses];
};

// Scalars that live on the device between kernels of one solve.
struct DevScalars {
  double t;            // FISTA t_k
  double beta;         // momentum factor of the current iteration
  double beta_used;    // the factor the last finalize applied to form y_{k+1}
  double restart_dot;  // Re<y_k - x_k, x_k - x_{k-1}> of the last iteration
  double rnorm2;       // ||H x - b||^2 of the last forward with a hologram
  double l1;           // ||x||_1 of the last objective evaluation
  double tv;           // TV(x) of the last objective evaluation
  int restart_flag;    // 1 if the last finalize restarted the momentum
  int nonfinite;       // sticky: a reduction saw NaN/Inf
  int accelerate;      // FISTA momentum on
  int restart;         // gradient restart enabled
};

// Reduction workspace: per-block partials and last-block tickets.
struct RedWork {
  double* partials;    // [4][kRedBlocks]
  unsigned* tickets;   // [8]
};

// ---------------------------------------------------------------------------
// FFT pass kernels (fft_kernels.cu)
// ---------------------------------------------------------------------------
enum RowIn { ROW_IN_C64 = 0, ROW_IN_F32 = 1, ROW_IN_STRIP = 2 };
enum RowOut { ROW_OUT_C64 = 0, ROW_OUT_STRIP = 1 };
enum RowEpi { ROW_EPI_SCALE = 0, ROW_EPI_GRAD = 1 };

struct RowArgs {
  const void* src;     // input planes (layout per RowIn)
  float2* dst;         // output planes (layout per RowOut)
  const float2* y;     // ROW_EPI_GRAD: volume y, row-major
  int nx, ny, nz;
  float scale;         // ROW_EPI_SCALE: out = scale * g; ROW_EPI_GRAD: v = y - scale * g
  FftPlan plan;        // along x
  const float2* tw;    // twiddles exp(-2 pi i m / nx), m < nx
  const int* occ;      // forward rows (complex input): [nz + 1] plane occupancy; when
                       // occ[nz] != 0, planes z with occ[z] == 0 are all zero and
                       // skipped (nothing written); null: every plane
  int teams;           // register engine: rows (transforms) per CTA, 1, 2, 4 or 8 (0: 4)
};

enum ColMode { COL_FWD_ZSUM = 0, COL_ADJ_GEN = 1, COL_PLAIN_FWD = 2, COL_PLAIN_INV = 3 };

struct ColArgs {
  const float2* src;
  float2* dst;
  const uint2* phase;  // [ny][nx] {phi0, phid}: plane j has phase phi0 + j*phid (2^-32 cycles)
  const float* amp;    // [ny][nx] 1 on the propagating band, 0 otherwise
  int nx, ny, nz;
  int z_per_group;     // planes per CTA along blockIdx.y
  float scale;
  FftPlan plan;        // along y
  const float2* tw;    // twiddles exp(-2 pi i m / ny), m < ny
  const int* occ;      // COL_FWD_ZSUM: [nz + 1] plane occupancy as for the rows; skipped
                       // planes are left out of the z-sum; null: every plane
};

cudaError_t launch_rows(int dir_inverse, int in, int out, int epi, const RowArgs& a,
                        cudaStream_t s);
cudaError_t launch_cols(int mode, const ColArgs& a, int groups, cudaStream_t s);
size_t rows_smem_bytes(int nx, int teams = 4);
constexpr int kRowTeams[4] = {1, 2, 4, 8};   // row-pass tile shapes the autotuner tries
size_t cols_smem_bytes(int mode, int ny);
bool reg_length(int n);   // lengths served by the register FFT engine
// Resident CTAs per SM of the forward column pass for this ny (sizes the z-groups).
int cols_ctas_per_sm(int ny);

// S = sum_g partial[g]; if bhat: out = S - bhat and ||out||^2 / (nx ny) -> sc->rnorm2.
cudaError_t launch_zsum(const float2* partial, int groups, const float2* bhat, float2* out,
                        int nx, int ny, DevScalars* sc, RedWork w, cudaStream_t s);
// After the forward of the iterate x_k (partials of its z-groups): S_x = F H x_k
// -> sx; ||S_x - F b||^2 / (nx ny) -> sc->rnorm2 (the data term of x_k); and, by
// linearity, the residual spectrum of y_{k+1} = x_k + beta (x_k - x_{k-1}) ->
// ry: S_x + beta (S_x - sx_prev) - F b with the beta the finalize used
// (sc->beta_used), or S_x - F b after a restart (sc->restart_flag).
cudaError_t launch_zsum_next(const float2* partial, int groups, const float2* bhat,
                             const float2* sx_prev, float2* sx, float2* ry, int nx, int ny,
                             DevScalars* sc, RedWork w, cudaStream_t s);

// ---------------------------------------------------------------------------
// TV / prox / FISTA kernels (tv_kernels.cu)
// ---------------------------------------------------------------------------
struct DevScalars;
struct TvArgs {
  CUtensorMap tm_v;    // v (see make_volume_tmap; box height per schedule)
  CUtensorMap tm_p[3]; // dual input p_x, p_y, p_z
  float2* pout[3];     // dual output (must not alias the input)
  int* err;            // set to 1 if a bounded wait gave up
  int nx, ny, nz, dims;
  int zchunk;
  // Two-step kernel only: with zchunk2 > 0 the tiles from split_tile on are
  // cut into z-chunks of zchunk2 planes and launched after the others, so
  // that shorter CTAs fill the last wave; zchunk2 = 0: every tile in
  // z-chunks of zchunk planes.
  int split_tile;
  int zchunk2;
  float mu;            // t_tv
  float step;          // 1 / (4 dims mu)
  // Fused finalize (the last two-step launch of a prox writes x = soft(v -
  // mu D^H p, kappa) instead of p; in FISTA mode also y_{k+1} and the
  // restart reduction, exactly as the finalize kernel).
  int fin_mode;        // FinMode
  float kappa;         // t_l1
  const float2* x_prev;
  const float2* y;
  float2* x_out;
  float2* y_out;
  DevScalars* sc;
  double* fin_partials;   // one double per CTA of the launch
  unsigned* fin_ticket;   // last-block counter (reset by the last block)
  int* occ;               // FISTA: [nz + 1], zeroed before the launch; occ[z] set for
                          // every plane z with a non-zero voxel of x_k or y_{k+1},
                          // occ[nz] = 1 if some plane has none; or null
  // Accelerated dual (FGP), one-step launches: the input dual (tm_p) is the
  // extrapolated r_k, pout receives p_k = Pi(r_k + step D u); pprev holds
  // p_{k-1} (not read on the first step, where it is zero); when rout[0] is
  // non-null it receives r_{k+1} = p_k + fgp_beta (p_k - p_{k-1}).
  const float2* pprev[3];
  float2* rout[3];
  float fgp_beta;
};
// nsteps = 1 or 2 dual steps in one launch; first: the input dual is zero;
// final (two-step launches only): fused finalize, no dual output.
cudaError_t launch_tv_step(bool first, int nsteps, const TvArgs& a, cudaStream_t s,
                           bool final = false, bool fgp = false);
// CTAs of a two-step launch with that z-chunking (final: the fused-finalize tile).
int tv2_ctas(int nx, int ny, int nz, bool final, int zchunk, int split_tile, int zchunk2);
// Box of box_rows x box_cols complex elements: (kTvBoxH1, kTvBoxW) for the
// one-step kernel, (kTv2BoxH, kTv2BoxW) for the two-step kernel.
cudaError_t make_volume_tmap(CUtensorMap* tm, const void* base, int nx, int ny, int nz,
                             int box_rows, int box_cols);

enum FinMode { FIN_PROX = 0, FIN_FISTA = 1 };
constexpr int kFinFistaOcc = 2;   // fused-finalize kernel variant: FISTA + plane occupancy
struct FinArgs {
  const float2* v;
  const float2* p[3];  // may be null (no TV): u = v
  const float2* x_prev;
  const float2* y;
  float2* x_out;
  float2* y_out;
  int nx, ny, nz, dims;
  float mu;            // t_tv
  float kappa;         // t_l1
  DevScalars* sc;
  RedWork w;
};
cudaError_t launch_finalize(int mode, const FinArgs& a, cudaStream_t s);
cudaError_t launch_restart_fixup(const float2* x, float2* y, size_t nvox, const DevScalars* sc,
                                 cudaStream_t s);
// F = sc->rnorm2 + lam_l1 * L1(x) + lam_tv * TV(x) -> *f_out (device double)
cudaError_t launch_objective(const float2* x, int nx, int ny, int nz, int dims, double lam_l1,
                             double lam_tv, DevScalars* sc, RedWork w, double* f_out,
                             cudaStream_t s);
cudaError_t launch_wait_selftest(int* flag, int polls, cudaStream_t s);
cudaError_t launch_init_scalars(DevScalars* sc, int accelerate, int restart, cudaStream_t s);

// ---------------------------------------------------------------------------
// FASTA-style solver (fasta_kernels.cu)
// ---------------------------------------------------------------------------
// v = x - tau g over n complex values.
cudaError_t launch_grad_step(const float2* x, const float2* g, float tau, float2* v, size_t n,
                             cudaStream_t s);
// out[0] = Re<a - b, c - d>, out[1] = ||a - b||^2, out[2] = ||c - d||^2 (d null: 0),
// FP64 on the device; uses partial rows 1-3 and ticket 4 of w.
cudaError_t launch_dots(const float2* a, const float2* b, const float2* c, const float2* d,
                        size_t n, RedWork w, double* out, cudaStream_t s);

// ---------------------------------------------------------------------------
// Detection (detect_kernels.cu)
// ---------------------------------------------------------------------------
struct DetectWork {
  int* label = nullptr;          // [nvox] union-find parent, -1 below threshold
  int* cid = nullptr;            // [nvox] compact component id, valid at roots
  unsigned* block_counts = nullptr;  // [nblocks] roots per 1024 voxels, then offsets
  unsigned* maxbits = nullptr;   // [1] max |x|^2 as float bits
  int* ncomp = nullptr;          // [1]
  double* stats = nullptr;       // [capacity][5]: sum w, sum w*i, sum w*j, sum w*k, count
  long long* first = nullptr;    // [capacity] smallest linear index
  size_t capacity = 0;
};
// Threshold, label, flatten, count roots; *ncomp_host receives the number of
// components (synchronises the stream). *err_dev is set if a union-find loop
// hit its bound.
cudaError_t detect_label(const float2* x, int nx, int ny, int nz, float rel, DetectWork& w,
                         int* err_dev, int* ncomp_host, cudaStream_t s);
// Component ids, first indices and FP64 sums for ncomp <= w.capacity components.
cudaError_t detect_stats(const float2* x, int nx, int ny, int nz, DetectWork& w, int ncomp,
                         cudaStream_t s);

// Detection on a per-plane COO form (work in proportion to the non-zeros).
struct CooDetectWork {
  long long* lin = nullptr;      // [capacity] linear indices of the entries above threshold
  float* wgt = nullptr;          // [capacity] their |x|
  int* label = nullptr;          // [capacity] union-find parents (list positions)
  int* cid = nullptr;            // [capacity] compact component id, valid at roots
  unsigned* block_counts = nullptr;  // [capacity / 1024 + 1]
  unsigned* maxbits = nullptr;   // [1]
  int* nhits = nullptr;          // [1]
  int* ncomp = nullptr;          // [1]
  size_t capacity = 0;           // entries (nnz) the buffers hold
};
// Threshold over the nnz > 0 listed values, compaction of the entries above
// it; *m_host receives their number (synchronises the stream).
cudaError_t detect_coo_hits(const long long* plane_off, const int* rows, const int* cols,
                            const float2* vals, long long nnz, int nx, int ny, int nz, float rel,
                            CooDetectWork& w, int* m_host, cudaStream_t s);
// Union-find over the m > 0 compacted entries; *ncomp_host receives the
// number of components (synchronises the stream).
cudaError_t detect_coo_label(int m, int nx, int ny, CooDetectWork& w, int* err_dev,
                             int* ncomp_host, cudaStream_t s);
// First indices and FP64 sums [ncomp][5] of the components.
cudaError_t detect_coo_stats(int m, int nx, int ny, CooDetectWork& w, int ncomp, double* stats,
                             long long* first, cudaStream_t s);

// ---------------------------------------------------------------------------
// Warm-start network convolutions (conv_kernels.cu)
// ---------------------------------------------------------------------------
struct ConvArgs {
  const __nv_bfloat16* x;   // [voxels][ck] (forward: input; dgrad: output gradient)
  const __nv_bfloat16* w_;  // W[c_out][27][c_in]
  const float* bias;        // [n] or null
  void* y;                  // [voxels][n], BF16 or FP32
  int d, h, w;              // volume (z, y, x) sizes
  int ck, n;                // gathered channels (K per tap), output channels (N)
  int relu, out_f32;
  int* err;
};
struct WgradArgs {
  const __nv_bfloat16* x;   // [voxels][cin]
  const __nv_bfloat16* gy;  // [voxels][cout]
  float* partial;           // [nsplit][cout][27][cin]
  int d, h, w, cin, cout;
  int nsplit;               // CTAs per 16-channel input chunk (grid.x)
  int tiles_per_split;      // 128 x 2 voxel tiles of one CTA
  int* err;
};
// Halo-tile geometry of the forward / input-gradient convolution.
constexpr int kConvTW = 128;                   // output voxels along x per CTA (MMA M)
constexpr int kConvTH = 2;                     // output rows (y) per CTA
constexpr int kConvHX = kConvTW + 2;           // halo width
constexpr int kConvHaloKu = 3 * (kConvTH + 2) * kConvHX * 16;   // bytes per 8-channel group
// each group's box is a TMA tile copy, whose shared-memory destination must
// sit on a 128-byte boundary (with 4 rows per CTA, 37,440 B, it would not)
static_assert(kConvHaloKu % 128 == 0, "conv halo boxes must start on 128-byte boundaries");
constexpr int kConvHaloBytes = 2 * kConvHaloKu;                 // 16 channels
constexpr int kConvMaxGroups = 32;             // 256 channels / 8
struct ConvMaps {
  CUtensorMap m[kConvMaxGroups];
};
cudaError_t launch_conv(bool dgrad, const ConvArgs& a, cudaStream_t s);
// Tiled tensor map (no interleave, no swizzle, 256-byte L2 promotion, zero
// fill out of bounds); rank <= 5, strides in bytes for dims 1..rank-1.
cudaError_t encode_tmap(CUtensorMap* tm, CUtensorMapDataType type, int rank, const void* base,
                        const cuuint64_t* dims, const cuuint64_t* strides, const cuuint32_t* box);
// CTAs per input-channel chunk and tiles per CTA of the weight gradient.
void wgrad_plan(int d, int h, int w, int cin, int sms, int* nsplit, int* tiles_per_split);
cudaError_t launch_wgrad(const WgradArgs& a, float* gw, cudaStream_t s);
size_t conv_smem_bytes(int ck, int n);

// ---------------------------------------------------------------------------
// Per-plane COO compaction (coo_kernels.cu)
// ---------------------------------------------------------------------------
constexpr int kCooSeg = 1024;   // voxels per counting / writing CTA
int coo_segments(int nx, int ny);
// counts [nz * segments] int, seg_off [nz * segments], plane_off [nz + 1] (int64)
cudaError_t launch_coo_count(const float2* x, int nx, int ny, int nz, int* counts, long long* seg_off,
                             long long* plane_off, cudaStream_t s);
cudaError_t launch_coo_write(const float2* x, int nx, int ny, int nz, const long long* seg_off,
                             int* rows, int* cols, float2* vals, cudaStream_t s);
// zero-fills x, then scatters; *bad = 1 if an entry lies outside the plane
cudaError_t launch_coo_scatter(const int* rows, const int* cols, const float2* vals,
                               const long long* plane_off, int nx, int ny, int nz, float2* x,
                               int* bad, cudaStream_t s);

}  // namespace rihv
