// C ABI of librihv: handle, scratch, transfer-function phase tables and the
// drivers that sequence the kernels of the forward model, its adjoint, the
// fused-lasso prox and FISTA (Section 2 of arXiv 1904.04884).
#include <cuda_runtime.h>
#include <unistd.h>

#include <algorithm>
#include <functional>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <queue>
#include <string>
#include <vector>

#include "rihv_internal.cuh"

using namespace rihv;

namespace {

thread_local std::string g_last_error;

}  // namespace

namespace rihv {

void set_global_error(const char* msg) { g_last_error = msg ? msg : ""; }

int pointer_device(const void* p) {
  cudaPointerAttributes at{};
  if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return kNotDevicePtr;
  }
  if (at.type == cudaMemoryTypeManaged) return kManagedPtr;
  if (at.type != cudaMemoryTypeDevice) return kNotDevicePtr;
  return at.device;
}

// Reads one byte of every page of a host buffer that a copy is about to read
// or write. The first device-to-host copy into pinned memory after seconds of
// GPU-only work ran at a fraction of the link's speed (40-260 ms instead of
// 11 ms for 2.15 GB, growing over the life of the process) until the CPU had
// touched those pages; touching them first takes about 1 ms for 2 GB. Device
// and managed memory are left alone; the reads do not change the buffer.
volatile unsigned g_touch_sink = 0;

void touch_host_pages(const void* p, size_t bytes) {
  if (!p || bytes == 0 || pointer_device(p) != kNotDevicePtr) return;
  static const size_t page = [] {
    const long s = sysconf(_SC_PAGESIZE);
    return s > 0 ? static_cast<size_t>(s) : static_cast<size_t>(4096);
  }();
  const volatile unsigned char* q = static_cast<const volatile unsigned char*>(p);
  const uintptr_t base = reinterpret_cast<uintptr_t>(p);
  unsigned acc = 0;
  for (size_t off = 0; off < bytes; off = ((base + off) / page + 1) * page - base) acc += q[off];
  acc += q[bytes - 1];
  g_touch_sink = acc;
}

int stream_device(const void* stream) {
  if (!stream) return kLegacyStream;
  int dev = -1;
  if (cudaStreamGetDevice(static_cast<cudaStream_t>(const_cast<void*>(stream)), &dev) !=
      cudaSuccess) {
    cudaGetLastError();
    return kNotDevicePtr;
  }
  return dev;
}

}  // namespace rihv

namespace {

constexpr int kNumStages = 10;
enum Stage {
  ST_FORWARD = 0, ST_ADJOINT = 1, ST_TV = 2, ST_FINAL = 3, ST_OBJECTIVE = 4, ST_DETECT = 5,
  ST_SETUP = 6,
  // sub-stages of ST_TV, one scope per launch: starting from p = 0, reading
  // p, and the launch with the fused finalize
  ST_TV_FIRST = 7, ST_TV_MID = 8, ST_TV_FINAL = 9
};
constexpr int kEventPool = 65536;   // two per stage scope; a full pool flushes (synchronises)

bool supported_n(int n) {
  if (n < 16 || n > kMaxN) return false;
  int m = n, twos = 0, threes = 0;
  while (m % 2 == 0) { m /= 2; ++twos; }
  while (m % 3 == 0) { m /= 3; ++threes; }
  return m == 1 && twos >= 3 && threes <= 1;
}

FftPlan make_plan(int n) {
  FftPlan p{};
  p.n = n;
  int m = n;
  while (m % 8 == 0) { p.radix[p.npass++] = 8; m /= 8; }
  if (m % 4 == 0) { p.radix[p.npass++] = 4; m /= 4; }
  if (m % 2 == 0) { p.radix[p.npass++] = 2; m /= 2; }
  if (m % 3 == 0) { p.radix[p.npass++] = 3; m /= 3; }
  return p;
}

double frac(double x) { return x - std::floor(x); }

uint32_t to_cycles32(double f) {
  // f in [0, 1) -> nearest multiple of 2^-32, wrapped
  const double s = std::floor(f * 4294967296.0 + 0.5);
  return static_cast<uint32_t>(static_cast<uint64_t>(s) & 0xFFFFFFFFull);
}

double fft_freq(int k, int n, double pitch) {
  const int kk = (k < n / 2) ? k : k - n;   // even n
  return static_cast<double>(kk) / (n * pitch);
}

}  // namespace

struct rihv_ctx {
  int nx = 0, ny = 0, nz = 0;
  double wavelength = 0, pitch = 0, z0 = 0, dz = 0;
  size_t nxy = 0, nvox = 0;
  cudaStream_t stream = nullptr;
  rihv_options opt{};
  int device = 0;
  int groups = 1, zpg = 1;
  int sms = 152;
  int tv_zchunk = 0;                 // planes per TV z-chunk; 0: tv_default_zchunk
  int row_teams = 0;                 // rows per CTA of the register row pass; 0: the default
  bool batch_chunks = false;         // being captured into a batched graph (see tv_steps)
  double* fin_partials = nullptr;    // one per CTA of a fused-finalize TV launch
  int fin_ctas = 0;                  // capacity of fin_partials
  // z-chunk splits of the two-step TV launches, by launch tile ([0] reading
  // p or first, [1] fused final), for the z-chunk they were computed for
  struct TvSplitCache {
    int zchunk = -1, split_tile = 0, zchunk2 = 0;
  } tv_split[2];
  double tau = 0;
  FftPlan plan_x{}, plan_y{};
  std::string err;

  // device buffers
  float2* tw_x = nullptr;
  float2* tw_y = nullptr;
  uint2* phase = nullptr;
  float* amp = nullptr;
  float2* inter = nullptr;     // strip-major intermediate [nz][nx/W][ny][W]
  float2* partial = nullptr;   // [groups][ny][nx]
  float2* spec = nullptr;      // [ny][nx] spectrum sum / residual spectrum
  float2* sx[2] = {nullptr, nullptr};   // [ny][nx] F H x_k of the last two iterates
  float2* bhat = nullptr;      // [ny][nx] F b
  float* holo = nullptr;       // [ny][nx]
  float2* x = nullptr;         // volumes
  float2* y = nullptr;
  float2* v = nullptr;
  float2* pa[3] = {nullptr, nullptr, nullptr};
  float2* pb[3] = {nullptr, nullptr, nullptr};
  float2* pc[3] = {nullptr, nullptr, nullptr};   // accelerated dual: p_k, p_{k-1} (allocated on use)
  float2* pd[3] = {nullptr, nullptr, nullptr};
  float2* fasta_g[2] = {nullptr, nullptr};      // FASTA: gradients at x_k and at the candidate
  float2* fasta_x = nullptr;                    // FASTA: candidate x_{k+1}
  double* fasta_dots = nullptr;                 // FASTA: inner products of the last test
  std::vector<double> fasta_taus;               // FASTA: accepted steps of the last solve
  int fasta_backtracks = 0;
  DevScalars* sc = nullptr;
  RedWork red{};
  double* trace = nullptr;     // device objective trace
  int trace_cap = 0;
  int* det_err = nullptr;
  int* coo_counts = nullptr;         // per-plane segment counts (COO compaction)
  long long* coo_seg_off = nullptr;  // their exclusive offsets
  int* coo_bad = nullptr;            // set by the COO scatter for an entry off the plane
  int* tv_err = nullptr;       // set by a TV kernel whose bounded wait gave up
  int* occ = nullptr;          // [nz] planes of x_k / y_{k+1} with a non-zero voxel
  CUtensorMap tm_pa[3][3], tm_pb[3][3];   // [one-step, two-step, fused-finalize box]
  DetectWork det{};
  CooDetectWork cdet{};
  std::vector<void*> allocs;

  // profiling
  int prof = 0;                      // 0 off, 1 stage events, 2 also per TV launch
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  struct Rec { int stage; int launches; cudaEvent_t a, b; };
  std::vector<Rec> recs;
  double stage_ms[kNumStages] = {0};
  long long stage_launches[kNumStages] = {0};
};

// A batch of handles solved together: one CUDA graph runs every handle's
// whole solve on its own branch (fork from a master stream, join back).
struct rihv_batch_st {
  std::vector<rihv_ctx*> hs;
  cudaStream_t master = nullptr;
  std::vector<cudaStream_t> branch;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraphExec_t exec = nullptr;
  // what the captured graph was built for
  int iters = -1;
  float l1 = -1.f, ltv = -1.f;
  bool warm = false;
  std::vector<rihv_options> opts;
  std::vector<int> tunes;            // zchunk, zpg, row teams per handle
  std::vector<std::vector<long long>> launches;   // per handle, per stage, per graph launch
  std::vector<int> checks;           // objective checks per handle per launch
  bool conditional = false;          // graph with per-hologram stop tests (IF nodes)
  int* done_dev = nullptr;           // per handle: iterations run by the last launch
  std::vector<int> done;             // host copy after the last launch
};

namespace {

rihv_status fail(rihv_ctx* h, rihv_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (h) h->err = buf;
  g_last_error = buf;
  return st;
}

#define CK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(h, RIHV_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                  __FILE__, __LINE__);                                                   \
  } while (0)

#define CKS(call)                      \
  do {                                 \
    rihv_status s_ = (call);           \
    if (s_ != RIHV_OK) return s_;      \
  } while (0)

template <typename T>
rihv_status dalloc(rihv_ctx* h, T** p, size_t count) {
  void* ptr = nullptr;
  cudaError_t e = cudaMalloc(&ptr, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(h, RIHV_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", count * sizeof(T),
                cudaGetErrorString(e));
  }
  h->allocs.push_back(ptr);
  *p = static_cast<T*>(ptr);
  return RIHV_OK;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

rihv_status check_dev(rihv_ctx* h, const void* p, const char* name) {
  if (!p) return fail(h, RIHV_ERR_INVALID_ARG, "%s is NULL", name);
  if (!aligned16(p)) return fail(h, RIHV_ERR_INVALID_ARG, "%s is not 16-byte aligned", name);
  const int where = pointer_device(p);
  if (where == kNotDevicePtr) return fail(h, RIHV_ERR_INVALID_ARG, "%s is not device memory", name);
  // device memory of another GPU would be read through peer access or fault:
  // the handle's kernels run on the device it was created on
  if (where != kManagedPtr && where != h->device)
    return fail(h, RIHV_ERR_INVALID_ARG, "%s lives on device %d, the handle on device %d", name,
                where, h->device);
  return RIHV_OK;
}

// ---- profiling -------------------------------------------------------------
struct StageScope {
  rihv_ctx* h;
  int stage;
  int launches;
  cudaEvent_t a = nullptr;
  // min_level: the profiling level at which this scope records events (the
  // per-launch TV scopes only at level 2: an event between two launches keeps
  // the second from starting while the first drains)
  StageScope(rihv_ctx* hh, int st, int nl, int min_level = 1)
      : h(hh), stage(st), launches(nl) {
    h->stage_launches[stage] += launches;
    if (h->prof < min_level) return;
    if (h->ev_used + 2 > h->ev_pool.size()) flush();
    a = h->ev_pool[h->ev_used++];
    cudaEventRecord(a, h->stream);
  }
  ~StageScope() {
    if (!a) return;
    cudaEvent_t b = h->ev_pool[h->ev_used++];
    cudaEventRecord(b, h->stream);
    h->recs.push_back({stage, 0, a, b});
  }
  void flush() {
    cudaStreamSynchronize(h->stream);
    for (auto& r : h->recs) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, r.a, r.b);
      h->stage_ms[r.stage] += ms;
    }
    h->recs.clear();
    h->ev_used = 0;
  }
};

// ---- stage drivers ----------------------------------------------------------
// Rows per CTA of the register row pass when neither the options nor the
// autotuner chose: 2 from length 512 up (three CTAs per SM), else 4.
int default_row_teams(int nx, int ny) { return (nx >= 512 && ny % 2 == 0) ? 2 : 4; }

RowArgs row_args(rihv_ctx* h, const void* src, float2* dst, int nz) {
  RowArgs a{};
  a.src = src;
  a.dst = dst;
  a.nx = h->nx;
  a.ny = h->ny;
  a.nz = nz;
  a.scale = 1.f;
  a.plan = h->plan_x;
  a.tw = h->tw_x;
  a.teams = h->opt.fft_rows_per_cta > 0 ? h->opt.fft_rows_per_cta
            : h->row_teams > 0           ? h->row_teams
                                         : default_row_teams(h->nx, h->ny);
  return a;
}

ColArgs col_args(rihv_ctx* h, const float2* src, float2* dst) {
  ColArgs a{};
  a.src = src;
  a.dst = dst;
  a.phase = h->phase;
  a.amp = h->amp;
  a.nx = h->nx;
  a.ny = h->ny;
  a.nz = h->nz;
  a.z_per_group = h->zpg;
  a.scale = 1.f;
  a.plan = h->plan_y;
  a.tw = h->tw_y;
  return a;
}

// Spectrum of the modelled hologram S = sum_j H_j F x_j; with bhat, the
// residual spectrum R = S - F b and ||Hx - b||^2 -> sc->rnorm2. With occ
// (plane occupancy of xin), planes marked 0 are all-zero and skipped.
rihv_status forward_spectrum(rihv_ctx* h, const float2* xin, const float2* bhat, float2* out,
                             const int* occ = nullptr) {
  StageScope sc(h, ST_FORWARD, 3);
  RowArgs ra = row_args(h, xin, h->inter, h->nz);
  ColArgs ca = col_args(h, h->inter, h->partial);
  ra.occ = occ;
  ca.occ = occ;
  CK(launch_rows(0, ROW_IN_C64, ROW_OUT_STRIP, ROW_EPI_SCALE, ra, h->stream));
  CK(launch_cols(COL_FWD_ZSUM, ca, h->groups, h->stream));
  CK(launch_zsum(h->partial, h->groups, bhat, out, h->nx, h->ny, h->sc, h->red, h->stream));
  return RIHV_OK;
}

// Forward of the iterate x_k (k = 0: x_0, in the set-up): F H x_k -> sx[k & 1],
// its data term ||H x_k - b||^2 -> sc->rnorm2, and the residual spectrum of
// y_{k+1} -> spec by linearity from F H x_k and F H x_{k-1} (the momentum and
// restart the finalize of iteration k applied). With occ, all-zero planes
// of x_k are skipped.
rihv_status forward_iterate(rihv_ctx* h, const float2* xin, int k, const int* occ) {
  StageScope sc(h, ST_FORWARD, 3);
  RowArgs ra = row_args(h, xin, h->inter, h->nz);
  ColArgs ca = col_args(h, h->inter, h->partial);
  ra.occ = occ;
  ca.occ = occ;
  CK(launch_rows(0, ROW_IN_C64, ROW_OUT_STRIP, ROW_EPI_SCALE, ra, h->stream));
  CK(launch_cols(COL_FWD_ZSUM, ca, h->groups, h->stream));
  CK(launch_zsum_next(h->partial, h->groups, h->bhat, h->sx[(k + 1) & 1], h->sx[k & 1], h->spec,
                      h->nx, h->ny, h->sc, h->red, h->stream));
  return RIHV_OK;
}

// Per-plane inverse propagation of the spectrum `spec`: with grad, out =
// y - scale * F^-1(conj(H_j) spec); otherwise out = scale * F^-1(conj(H_j) spec).
rihv_status adjoint_planes(rihv_ctx* h, const float2* spec, const float2* y, float2* out,
                           float scale, bool grad) {
  StageScope sc(h, ST_ADJOINT, 2);
  CK(launch_cols(COL_ADJ_GEN, col_args(h, spec, h->inter), h->groups, h->stream));
  RowArgs ra = row_args(h, h->inter, out, h->nz);
  ra.scale = scale;
  ra.y = y;
  CK(launch_rows(1, ROW_IN_STRIP, ROW_OUT_C64, grad ? ROW_EPI_GRAD : ROW_EPI_SCALE, ra, h->stream));
  return RIHV_OK;
}

// 2D FFT of one plane (complex or real row-major input) -> row-major spectrum.
rihv_status fft2_plane(rihv_ctx* h, const void* src, bool real_in, float2* out) {
  CK(launch_rows(0, real_in ? ROW_IN_F32 : ROW_IN_C64, ROW_OUT_STRIP, ROW_EPI_SCALE,
                 row_args(h, src, h->inter, 1), h->stream));
  CK(launch_cols(COL_PLAIN_FWD, col_args(h, h->inter, out), 1, h->stream));
  return RIHV_OK;
}

// TV launch geometry (host policy; the kernels take the chunk as an argument).
// CTAs of a fused-final TV launch for a z-chunk.
int tv_final_ctas(int nx, int ny, int nz, int zchunk) {
  return ((nx + kTv2TxF - 1) / kTv2TxF) * ((ny + kTv2TyF - 1) / kTv2TyF) * ((nz + zchunk - 1) / zchunk);
}


// Planes per z-chunk of a TV launch when none was tuned (final: the
// fused-finalize launch's tile).
int tv_default_zchunk(int nx, int ny, int nz, int nsteps, int sms, bool final = false) {
  if (nsteps != 2) return 32;
  // One CTA per SM; a chunk of zc planes takes zc + 3 plane ticks (zc + 4 for
  // the fused final launch, one more plane of z halo). The cost of a chunk
  // size is (waves, rounded up) x (ticks per chunk), over chunks in [8, 256].
  // Every chunk also reads its z halo again, which this count leaves out, so
  // among the chunks within 3 % of the lowest cost the largest is taken.
  const int tx = final ? kTv2TxF : kTv2Tx, ty = final ? kTv2TyF : kTv2Ty;
  const int halo = final ? 4 : 3;
  const long tiles = static_cast<long>((nx + tx - 1) / tx) * ((ny + ty - 1) / ty);
  auto cost = [&](int c) {
    const long ctas = tiles * ((nz + c - 1) / c);
    return ((ctas + sms - 1) / sms) * (c + halo);
  };
  const int cmax = nz < kTvMaxChunk ? nz : kTvMaxChunk;
  const int cmin = nz < 8 ? nz : 8;
  long lowest = -1;
  for (int c = cmin; c <= cmax; ++c)
    if (lowest < 0 || cost(c) < lowest) lowest = cost(c);
  int best = cmin;
  for (int c = cmin; c <= cmax; ++c)
    if (cost(c) * 100 <= lowest * 103) best = c;
  return best;
}

// Split of a two-step TV launch (TvArgs::split_tile, zchunk2). With one CTA
// per SM, equal z-chunks leave the last wave partly idle (at 1024x1024x256,
// 1,152 CTAs fill 7.6 waves). Model: a CTA of c planes takes c + halo plane
// ticks and CTAs start in launch order on the first free SM. The last r
// tiles are cut into m = 2, 3 or 4 z-chunks (of at least 8 planes) and
// launched after the rest; the split with the shortest modelled makespan is
// taken if it saves at least 2 % over equal chunks.
void tv_choose_split(int ntiles, int nz, int zc, int halo, int sms, int* split_tile,
                     int* zchunk2) {
  *split_tile = 0;
  *zchunk2 = 0;
  auto makespan = [&](int ka, int zc2) {
    std::priority_queue<long, std::vector<long>, std::greater<long>> q;
    for (int i = 0; i < sms; ++i) q.push(0);
    auto run = [&](int tiles, int c) {
      for (int z0 = 0; z0 < nz; z0 += c) {
        const long len = std::min(c, nz - z0) + halo;
        for (int t = 0; t < tiles; ++t) {
          const long f = q.top();
          q.pop();
          q.push(f + len);
        }
      }
    };
    run(ka, zc);
    if (zc2 > 0) run(ntiles - ka, zc2);
    long m = 0;
    for (; !q.empty(); q.pop()) m = std::max(m, q.top());
    return m;
  };
  const long base = makespan(ntiles, 0);
  long best = base;
  const int rmax = std::min(ntiles, 2 * sms), rstep = std::max(1, sms / 64);
  for (int parts = 2; parts <= 4; ++parts) {
    const int zc2 = (zc + parts - 1) / parts;
    if (zc2 < 8) break;
    for (int r = rstep; r <= rmax; r += rstep) {
      const long m = makespan(ntiles - r, zc2);
      if (m < best) {
        best = m;
        *split_tile = ntiles - r;
        *zchunk2 = zc2;
      }
    }
  }
  if (best * 100 > base * 98) {
    *split_tile = 0;
    *zchunk2 = 0;
  }
}

// Planes per z-chunk of a TV launch of n dual steps in a prox of `per` steps
// per launch: the option, else (fused-final launch) its own tile's default,
// else the tuned chunk, else the default of the launch's tile (one-step
// launches: 32). In a batched graph the branches run concurrently, so the
// two-step launches take the largest chunk (fewest halo planes read twice)
// rather than the one that fills the waves of a lone launch. The fused-final
// launch keeps the lone-solve chunk: its restart-product partials follow the
// chunking, and with them a batched solve stays bitwise equal to a single one
// (no other TV result depends on the chunk).
int tv_launch_zchunk(const rihv_ctx* h, int n, int per, bool fused_last) {
  if (h->opt.tv_zchunk > 0) return std::min(h->opt.tv_zchunk, h->nz);
  if (fused_last) return tv_default_zchunk(h->nx, h->ny, h->nz, 2, h->sms, true);
  if (h->tv_zchunk > 0) return h->tv_zchunk;
  if (n != per) return 32;
  return (h->batch_chunks && per == 2) ? std::min(h->nz, kTvMaxChunk)
                                       : tv_default_zchunk(h->nx, h->ny, h->nz, per, h->sms);
}

// The split for a two-step launch of this handle (cached per tile and chunk).
void tv_split_for(rihv_ctx* h, bool final, int zc, int* split_tile, int* zchunk2) {
  auto& c = h->tv_split[final ? 1 : 0];
  if (c.zchunk != zc) {
    const int tx = final ? kTv2TxF : kTv2Tx, ty = final ? kTv2TyF : kTv2Ty;
    const int ntiles = ((h->nx + tx - 1) / tx) * ((h->ny + ty - 1) / ty);
    tv_choose_split(ntiles, h->nz, zc, final ? 4 : 3, h->sms, &c.split_tile, &c.zchunk2);
    c.zchunk = zc;
  }
  *split_tile = c.split_tile;
  *zchunk2 = c.zchunk2;
}

// K steps of the accelerated dual (FGP), one per launch: the step at the
// extrapolated dual r_k (held in pa / pb, read by TMA) writes p_k (pc / pd)
// and r_{k+1}; t_k and the extrapolation factors are computed here in FP64.
// Returns the buffer set holding p_K.
rihv_status tv_steps_fgp(rihv_ctx* h, const float2* v, float mu, int k, float2* const** pfinal) {
  if (!h->pc[0]) return fail(h, RIHV_ERR_INVALID_ARG, "accelerated dual scratch not allocated");
  StageScope sc(h, ST_TV, k);
  TvArgs a{};
  CK(make_volume_tmap(&a.tm_v, v, h->nx, h->ny, h->nz, kTvBoxH1, kTvBoxW));
  a.err = h->tv_err;
  a.nx = h->nx;
  a.ny = h->ny;
  a.nz = h->nz;
  a.dims = h->opt.tv_dims;
  a.zchunk = h->opt.tv_zchunk > 0 ? std::min(h->opt.tv_zchunk, h->nz) : 32;
  a.mu = mu;
  a.step = 1.f / (4.f * a.dims * mu);
  float2** ps[2] = {h->pc, h->pd};
  bool src_is_b = true;
  double t = 1.0;
  for (int i = 0; i < k; ++i) {
    const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
    a.fgp_beta = static_cast<float>((t - 1.0) / tn);
    t = tn;
    float2** rdst = src_is_b ? h->pa : h->pb;
    for (int c = 0; c < 3; ++c) {
      a.tm_p[c] = src_is_b ? h->tm_pb[0][c] : h->tm_pa[0][c];
      a.pout[c] = ps[i & 1][c];
      a.pprev[c] = i > 0 ? ps[(i - 1) & 1][c] : nullptr;
      a.rout[c] = i + 1 < k ? rdst[c] : nullptr;
    }
    {
      StageScope sub(h, i == 0 ? ST_TV_FIRST : ST_TV_MID, 1, 2);
      CK(launch_tv_step(i == 0, 1, a, h->stream, false, true));
    }
    src_is_b = !src_is_b;
  }
  *pfinal = ps[(k - 1) & 1];
  return RIHV_OK;
}

// K dual steps; returns the buffer set holding the final p. With `fin` (two
// steps per launch, K >= 2) the last launch also runs the finalize and
// *pfinal is null.
rihv_status tv_steps(rihv_ctx* h, const float2* v, float mu, int k, float2* const** pfinal,
                     const FinArgs* fin = nullptr, int fin_mode = FIN_PROX) {
  if (h->opt.tv_fgp) return tv_steps_fgp(h, v, mu, k, pfinal);
  // With tv_steps_per_launch = 2, two dual steps per launch; an odd K starts
  // with a single-step launch, so that the last launch is always a pair.
  const int per = h->opt.tv_steps_per_launch;
  const int launches = per == 2 ? k / 2 + (k % 2) : k;
  const bool fused = fin && per == 2 && k >= 2;
  StageScope sc(h, ST_TV, launches);
  CUtensorMap tm_v[3];
  CK(make_volume_tmap(&tm_v[0], v, h->nx, h->ny, h->nz, kTvBoxH1, kTvBoxW));
  if (per == 2) CK(make_volume_tmap(&tm_v[1], v, h->nx, h->ny, h->nz, kTv2BoxH, kTv2BoxW));
  if (fused) CK(make_volume_tmap(&tm_v[2], v, h->nx, h->ny, h->nz, kTv2BoxHF, kTv2BoxW));
  TvArgs a{};
  a.err = h->tv_err;
  a.nx = h->nx;
  a.ny = h->ny;
  a.nz = h->nz;
  a.dims = h->opt.tv_dims;
  a.mu = mu;
  a.step = 1.f / (4.f * a.dims * mu);
  if (fused) {
    a.fin_mode = fin_mode;
    a.kappa = fin->kappa;
    a.x_prev = fin->x_prev;
    a.y = fin->y;
    a.x_out = fin->x_out;
    a.y_out = fin->y_out;
    a.sc = fin->sc;
    a.fin_partials = h->fin_partials;
    a.fin_ticket = h->red.tickets + 3;
    if (fin_mode == FIN_FISTA && h->opt.skip_empty_planes) a.occ = h->occ;
  }
  float2** src = h->pb;
  float2** dst = h->pa;
  bool src_is_b = true;
  int done = 0;
  while (done < k) {
    const int n = (per == 2 && !(done == 0 && k % 2 == 1)) ? 2 : 1;
    const bool last = done + n == k;
    const int b = n == 2 ? ((fused && last) ? 2 : 1) : 0;
    // the fused-finalize launch has its own tile, so its own default chunk
    a.zchunk = tv_launch_zchunk(h, n, per, fused && last);
    // two-step launches: shorter z-chunks for the last tiles where that fills
    // the last wave (not for the other launches of a batched graph, whose
    // branches fill the GPU together; the fused-final launch's split depends
    // only on the shape, so a batched solve keeps its restart-product order)
    a.split_tile = 0;
    a.zchunk2 = 0;
    if (n == 2 && h->opt.tv_split && ((fused && last) || !h->batch_chunks))
      tv_split_for(h, fused && last, a.zchunk, &a.split_tile, &a.zchunk2);
    if (fused && last &&
        (tv2_ctas(h->nx, h->ny, h->nz, true, a.zchunk, a.split_tile, a.zchunk2) > h->fin_ctas ||
         a.zchunk > kTvMaxChunk))
      return fail(h, RIHV_ERR_INVALID_ARG, "z-chunk outside the fused finalize's range");
    a.tm_v = tm_v[b];
    for (int c = 0; c < 3; ++c) {
      a.tm_p[c] = src_is_b ? h->tm_pb[b][c] : h->tm_pa[b][c];
      a.pout[c] = dst[c];
    }
    if (fused && last && a.occ)
      CK(cudaMemsetAsync(a.occ, 0, sizeof(int) * (h->nz + 1), h->stream));
    {
      StageScope sub(h, (fused && last) ? ST_TV_FINAL : (done == 0 ? ST_TV_FIRST : ST_TV_MID), 1, 2);
      CK(launch_tv_step(done == 0, n, a, h->stream, fused && last));
    }
    done += n;
    std::swap(src, dst);
    src_is_b = !src_is_b;
  }
  *pfinal = fused ? nullptr : src;
  return RIHV_OK;
}

rihv_status prox_into(rihv_ctx* h, const float2* v, float t_l1, float t_tv, int k, int mode,
                      float2* x_out) {
  float2* const* pf = nullptr;
  const bool tv = (t_tv > 0.f && k > 0);
  FinArgs f{};
  f.v = v;
  f.x_prev = h->x;
  f.y = h->y;
  f.x_out = x_out;
  f.y_out = h->y;
  f.nx = h->nx;
  f.ny = h->ny;
  f.nz = h->nz;
  f.dims = h->opt.tv_dims;
  f.mu = tv ? t_tv : 0.f;
  f.kappa = t_l1;
  f.sc = h->sc;
  f.w = h->red;
  if (tv) CKS(tv_steps(h, v, t_tv, k, &pf, h->opt.fuse_finalize ? &f : nullptr, mode));
  if (!tv || pf) {
    StageScope sc(h, ST_FINAL, mode == FIN_FISTA ? 2 : 1);
    for (int c = 0; c < 3; ++c) f.p[c] = tv ? pf[c] : nullptr;
    CK(launch_finalize(mode, f, h->stream));
    if (mode == FIN_FISTA) CK(launch_restart_fixup(x_out, h->y, h->nvox, h->sc, h->stream));
  } else if (mode == FIN_FISTA) {
    StageScope sc(h, ST_FINAL, 1);
    CK(launch_restart_fixup(x_out, h->y, h->nvox, h->sc, h->stream));
  }
  return RIHV_OK;
}

constexpr int kMaxGroups = 32;

void choose_groups(rihv_ctx* h, int nz) {
  const int strips = h->nx / kStrip;
  const double slots = static_cast<double>(cols_ctas_per_sm(h->ny)) * h->sms;
  int best_zpg = nz;
  double best_eff = -1.0;
  for (int zpg = nz; zpg >= 1; --zpg) {
    const int g = (nz + zpg - 1) / zpg;
    if (g > kMaxGroups) break;
    const double waves = strips * g / slots;
    const double eff = waves < 1.0 ? waves : waves / std::ceil(waves);
    if (eff > best_eff + 0.03) {
      best_eff = eff;
      best_zpg = zpg;
    }
  }
  h->zpg = best_zpg;
  h->groups = (nz + best_zpg - 1) / best_zpg;
}

// Whether a FISTA iteration with TV weight t_tv (already times the step)
// leaves the plane occupancy of x_k and y_{k+1} in h->occ: only the fused
// finalize records it, and only the register FFT engine reads it.
bool occ_tracked(const rihv_ctx* h, float t_tv) {
  const int k = h->opt.n_inner;
  return h->opt.skip_empty_planes && h->opt.fuse_finalize && h->opt.tv_steps_per_launch == 2 &&
         t_tv > 0.f && k >= 2 && reg_length(h->nx) && reg_length(h->ny);
}

rihv_status copy_in(rihv_ctx* h, void* dst, const void* src, size_t bytes) {
  touch_host_pages(src, bytes);
  CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, h->stream));
  return RIHV_OK;
}

rihv_status check_solve_args(rihv_ctx* h, float l1, float ltv, int iters) {
  if (iters < 0 || !(l1 >= 0.f) || !(ltv >= 0.f) || !std::isfinite(l1) || !std::isfinite(ltv))
    return fail(h, RIHV_ERR_INVALID_ARG, "iters >= 0 and finite lambdas >= 0 required");
  return RIHV_OK;
}

rihv_status ensure_trace(rihv_ctx* h, int nchecks) {
  if (nchecks <= h->trace_cap) return RIHV_OK;
  if (h->trace) cudaFree(h->trace);
  h->trace = nullptr;
  h->trace_cap = 0;
  if (cudaMalloc(&h->trace, sizeof(double) * nchecks) != cudaSuccess) {
    cudaGetLastError();
    return fail(h, RIHV_ERR_OOM, "trace allocation failed");
  }
  h->trace_cap = nchecks;
  return RIHV_OK;
}

// End of a chunk of FISTA iterations inside a batched graph: records the
// iterations run and, if a chunk follows, sets its IF condition: stop once
// the objective just computed is <= the threshold (rihv_solve's test).
__global__ void k_chunk_end(int* done, int k_end, const double* f, double thr,
                            cudaGraphConditionalHandle next, int has_next) {
  *done = k_end;
  if (has_next) {
    const double v = *f;
    cudaGraphSetConditional(next, (v <= thr) ? 0u : 1u);
  }
}

cudaError_t launch_chunk_end(int* done, int k_end, const double* f, double thr,
                             cudaGraphConditionalHandle next, int has_next, cudaStream_t s) {
  k_chunk_end<<<1, 1, 0, s>>>(done, k_end, f, thr, next, has_next && f ? 1 : 0);
  return cudaGetLastError();
}

// Solve set-up from the hologram already in h->holo: F b, x_0 (zero unless
// warm, in which case h->x already holds it), y_1 = x_0, scalars, flags, and
// the forward of x_0.
rihv_status enqueue_setup(rihv_ctx* h, bool warm) {
  StageScope sc(h, ST_SETUP, 3);
  CKS(fft2_plane(h, h->holo, true, h->bhat));
  const size_t vb = h->nvox * sizeof(float2);
  if (!warm) CK(cudaMemsetAsync(h->x, 0, vb, h->stream));
  CK(cudaMemcpyAsync(h->y, h->x, vb, cudaMemcpyDeviceToDevice, h->stream));
  CK(launch_init_scalars(h->sc, h->opt.accelerate, h->opt.restart, h->stream));
  CK(cudaMemsetAsync(h->tv_err, 0, sizeof(int), h->stream));
  // F H x_0, and the residual spectrum of y_1 = x_0
  CKS(forward_iterate(h, h->x, 0, nullptr));
  return RIHV_OK;
}

// FISTA iteration k (1-based): gradient step from the residual spectrum of
// y_k, fused-lasso prox with momentum and restart, then the forward of x_k
// (one forward per iteration: it gives F(x_k)'s data term and, by linearity,
// the residual of y_{k+1}); every check_every iterations the objective F(x_k)
// goes to trace slot *check, which is then incremented.
rihv_status enqueue_iteration(rihv_ctx* h, int k, float lambda_l1, float lambda_tv, int* check) {
  const float tau = static_cast<float>(h->tau);
  const float grad_scale = static_cast<float>(2.0 * h->tau / static_cast<double>(h->nxy));
  // (c) v = y - tau * 2 H^H r, with R = F(H y_k - b) in spec (left there by
  // the forward of the previous iterate, or by the set-up)
  CKS(adjoint_planes(h, h->spec, h->y, h->v, grad_scale, true));
  // (d) x_k = prox(v), momentum, restart
  CKS(prox_into(h, h->v, tau * lambda_l1, tau * lambda_tv, h->opt.n_inner, FIN_FISTA, h->x));
  // (a) forward of x_k: the data term of F(x_k) and R = F(H y_{k+1} - b) for
  // the next iteration; with the empty-plane skip, all-zero planes of x_k
  // are left out
  const int* occ = occ_tracked(h, tau * lambda_tv) ? h->occ : nullptr;
  CKS(forward_iterate(h, h->x, k, occ));
  const int M = h->opt.check_every;
  if (M > 0 && k % M == 0) {
    StageScope sc(h, ST_OBJECTIVE, 1);
    CK(launch_objective(h->x, h->nx, h->ny, h->nz, h->opt.tv_dims, lambda_l1, lambda_tv, h->sc,
                        h->red, h->trace + *check, h->stream));
    ++*check;
  }
  return RIHV_OK;
}

// Per-component sums and first indices for ncomp components (grown on demand).
rihv_status ensure_stats(rihv_ctx* h, int ncomp) {
  DetectWork& w = h->det;
  if (static_cast<size_t>(ncomp) <= w.capacity) return RIHV_OK;
  if (w.stats) cudaFree(w.stats);
  if (w.first) cudaFree(w.first);
  w.stats = nullptr;
  w.first = nullptr;
  w.capacity = 0;
  const size_t cap = std::max<size_t>(ncomp, 1024);
  if (cudaMalloc(&w.stats, cap * 5 * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&w.first, cap * sizeof(long long)) != cudaSuccess) {
    cudaGetLastError();
    return fail(h, RIHV_ERR_OOM, "detection stats allocation failed");
  }
  w.capacity = cap;
  return RIHV_OK;
}

// Reads the ncomp components' sums back, drops those of <= min_vox voxels and
// writes the rest (in component order, i.e. by smallest voxel index).
rihv_status emit_particles(rihv_ctx* h, int ncomp, int min_vox, rihv_particle* out, int max_out,
                           int* n_out) {
  std::vector<double> st(static_cast<size_t>(ncomp) * 5);
  std::vector<long long> first(ncomp);
  int err = 0;
  if (ncomp > 0) {
    CK(cudaMemcpyAsync(st.data(), h->det.stats, st.size() * sizeof(double),
                       cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(first.data(), h->det.first, first.size() * sizeof(long long),
                       cudaMemcpyDeviceToHost, h->stream));
  }
  CK(cudaMemcpyAsync(&err, h->det_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (err) return fail(h, RIHV_ERR_TIMEOUT, "union-find exceeded its iteration bound");
  int n = 0;
  for (int c = 0; c < ncomp; ++c) {
    const double* s = &st[static_cast<size_t>(c) * 5];
    const int cnt = static_cast<int>(s[4] + 0.5);
    if (cnt <= min_vox) continue;
    if (n < max_out) {
      rihv_particle& p = out[n];
      p.cx = s[1] / s[0];
      p.cy = s[2] / s[0];
      p.cz = s[3] / s[0];
      p.weight = s[0];
      p.first = first[c];
      p.nvox = cnt;
      p.pad_ = 0;
    }
    ++n;
  }
  *n_out = n;
  return RIHV_OK;
}

// Forward-backward splitting with FASTA's adaptive spectral step and
// non-monotone backtracking (the option solver = 1). The hologram is in
// h->holo and, if warm, x_0 in h->x. Per iteration: v = x_k - tau g_k, the
// fused-lasso prox of v (step tau) into the candidate, its forward (data term
// f and residual spectrum), then Re<dx, g_k> and ||dx||^2 on the device; the
// host accepts the candidate when f <= max of the last 10 f + Re<dx, g_k> +
// ||dx||^2 / (2 tau) (up to 1e-6 of that maximum) or halves tau and retries
// (at most 20 times). After acceptance g_{k+1} = 2 H^H r_{k+1} and the next
// step from <dx, dg>, ||dx||^2, ||dg||^2: tau_m = <dx,dg>/||dg||^2, tau_s =
// ||dx||^2/<dx,dg>, tau = tau_m if 2 tau_m > tau_s else tau_s - tau_m/2, or
// 1.5 tau when <dx,dg> <= 0. Two host synchronisations per iteration.
rihv_status solve_fasta(rihv_ctx* h, bool warm, float l1, float ltv, int iters, int* check_out,
                        int* done_out) {
  if (!h->fasta_g[0]) return fail(h, RIHV_ERR_INVALID_ARG, "FASTA scratch not allocated");
  const size_t vb = h->nvox * sizeof(float2);
  // The accepted candidate swaps buffers with x. Graphs captured earlier hold
  // the address of h->x, so it is handed back on every return (with the
  // result copied into it on success).
  struct XHome {
    rihv_ctx* h;
    float2* home;
    ~XHome() {
      if (h->x != home) std::swap(h->x, h->fasta_x);
    }
  } x_home{h, h->x};
  const float gscale = static_cast<float>(2.0 / static_cast<double>(h->nxy));
  CKS(fft2_plane(h, h->holo, true, h->bhat));
  if (!warm) CK(cudaMemsetAsync(h->x, 0, vb, h->stream));
  CK(launch_init_scalars(h->sc, 0, 0, h->stream));
  CK(cudaMemsetAsync(h->tv_err, 0, sizeof(int), h->stream));
  int cur = 0;
  CKS(forward_spectrum(h, h->x, h->bhat, h->spec));
  CKS(adjoint_planes(h, h->spec, nullptr, h->fasta_g[cur], gscale, false));
  DevScalars hs{};
  CK(cudaMemcpyAsync(&hs, h->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  std::vector<double> f_hist = {hs.rnorm2};
  double tau = h->tau;
  h->fasta_taus.clear();
  h->fasta_backtracks = 0;
  const int M = h->opt.check_every;
  const bool stop_test = h->opt.f_star > 0.0 && M > 0;
  int check = 0, done = 0;
  double dots[3];
  for (int k = 1; k <= iters; ++k) {
    double f_new = 0.0;
    for (int bt = 0;; ++bt) {
      CK(launch_grad_step(h->x, h->fasta_g[cur], static_cast<float>(tau), h->v, h->nvox, h->stream));
      CKS(prox_into(h, h->v, static_cast<float>(tau) * l1, static_cast<float>(tau) * ltv,
                    h->opt.n_inner, FIN_PROX, h->fasta_x));
      CKS(forward_spectrum(h, h->fasta_x, h->bhat, h->spec));
      CK(launch_dots(h->fasta_x, h->x, h->fasta_g[cur], nullptr, h->nvox, h->red, h->fasta_dots,
                     h->stream));
      CK(cudaMemcpyAsync(dots, h->fasta_dots, 3 * sizeof(double), cudaMemcpyDeviceToHost,
                         h->stream));
      CK(cudaMemcpyAsync(&hs, h->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
      f_new = hs.rnorm2;
      if (!std::isfinite(f_new) || !std::isfinite(dots[0]) || !std::isfinite(dots[1]))
        return fail(h, RIHV_ERR_NONFINITE, "FASTA step produced NaN or Inf");
      const size_t w0 = f_hist.size() > 10 ? f_hist.size() - 10 : 0;
      const double f_max = *std::max_element(f_hist.begin() + w0, f_hist.end());
      const double bound = f_max + dots[0] + dots[1] / (2.0 * tau);
      if (f_new <= bound + 1e-6 * std::fabs(f_max) || bt == 20) break;
      tau *= 0.5;
      ++h->fasta_backtracks;
    }
    h->fasta_taus.push_back(tau);
    const int nxt = cur ^ 1;
    CKS(adjoint_planes(h, h->spec, nullptr, h->fasta_g[nxt], gscale, false));
    CK(launch_dots(h->fasta_x, h->x, h->fasta_g[nxt], h->fasta_g[cur], h->nvox, h->red,
                   h->fasta_dots, h->stream));
    CK(cudaMemcpyAsync(dots, h->fasta_dots, 3 * sizeof(double), cudaMemcpyDeviceToHost,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    double tau_next = 0.0;
    if (dots[0] > 0.0) {
      const double tau_s = dots[1] / dots[0];
      const double tau_m = dots[0] / dots[2];
      tau_next = (2.0 * tau_m > tau_s) ? tau_m : tau_s - 0.5 * tau_m;
    }
    tau = (tau_next > 0.0 && std::isfinite(tau_next)) ? tau_next : 1.5 * tau;
    std::swap(h->x, h->fasta_x);
    cur = nxt;
    f_hist.push_back(f_new);
    done = k;
    if (M > 0 && k % M == 0) {
      // the data term of x_k is the last forward's (sc->rnorm2)
      CK(launch_objective(h->x, h->nx, h->ny, h->nz, h->opt.tv_dims, l1, ltv, h->sc, h->red,
                          h->trace + check, h->stream));
      ++check;
      if (stop_test) {
        double f = 0;
        CK(cudaMemcpyAsync(&f, h->trace + check - 1, sizeof(double), cudaMemcpyDeviceToHost,
                           h->stream));
        CK(cudaStreamSynchronize(h->stream));
        if (f <= h->opt.f_star * (1.0 + h->opt.tol)) break;
      }
    }
  }
  if (h->x != x_home.home)
    CK(cudaMemcpyAsync(x_home.home, h->x, vb, cudaMemcpyDeviceToDevice, h->stream));
  *check_out = check;
  *done_out = done;
  return RIHV_OK;
}

// After the stream has finished: TV wait failures and non-finite reductions.
rihv_status read_solve_errors(rihv_ctx* h) {
  DevScalars hs{};
  int tv_err = 0;
  CK(cudaMemcpy(&hs, h->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(&tv_err, h->tv_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (tv_err) return fail(h, RIHV_ERR_TIMEOUT, "a TV kernel's bounded wait gave up");
  if (hs.nonfinite) return fail(h, RIHV_ERR_NONFINITE, "a reduction produced NaN or Inf");
  return RIHV_OK;
}

}  // namespace

// =============================================================================
// C ABI
// =============================================================================
extern "C" {

void rihv_default_options(rihv_options* o) {
  if (!o) return;
  o->tv_dims = 3;
  o->restart = 1;
  o->accelerate = 1;
  o->n_inner = 20;
  o->check_every = 10;
  o->tol = 0.0;
  o->f_star = 0.0;
  o->tv_steps_per_launch = 2;
  o->fuse_finalize = 1;
  o->skip_empty_planes = 0;
  o->tv_zchunk = 0;
  o->fft_rows_per_cta = 0;
  o->tv_fgp = 0;
  o->tv_split = 1;
  o->solver = 0;
}

const char* rihv_last_error(rihv_handle h) {
  return h ? h->err.c_str() : g_last_error.c_str();
}

rihv_status rihv_create(int nx, int ny, int nz, double wavelength, double pitch, double z0,
                        double dz, rihv_handle* out) {
  rihv_ctx* h = nullptr;
  if (!out) return fail(nullptr, RIHV_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!supported_n(nx) || !supported_n(ny) || nz < 1 || nz > 4096)
    return fail(nullptr, RIHV_ERR_UNSUPPORTED_SIZE,
                "unsupported size %dx%dx%d (nx, ny in 2^a 3^b, 16..1024, a>=3, b<=1; 1<=nz<=4096)",
                nx, ny, nz);
  if (!(wavelength > 0) || !(pitch > 0) || !std::isfinite(z0) || !std::isfinite(dz))
    return fail(nullptr, RIHV_ERR_INVALID_ARG, "wavelength and pitch must be > 0, z0/dz finite");
  h = new (std::nothrow) rihv_ctx();
  if (!h) return fail(nullptr, RIHV_ERR_OOM, "host allocation failed");
  h->nx = nx; h->ny = ny; h->nz = nz;
  h->wavelength = wavelength; h->pitch = pitch; h->z0 = z0; h->dz = dz;
  h->nxy = static_cast<size_t>(nx) * ny;
  h->nvox = h->nxy * nz;
  rihv_default_options(&h->opt);
  h->plan_x = make_plan(nx);
  h->plan_y = make_plan(ny);
  cudaGetDevice(&h->device);

  // z-groups of the column passes: the fewest groups whose grid fills whole
  // waves of the resident slots (2 CTAs per SM) to within 3 %, at most 32.
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  h->sms = sms;
  choose_groups(h, nz);

  auto cleanup = [&](rihv_status st) {
    rihv_destroy(h);
    return st;
  };
  rihv_status st;
#define AL(ptr, n) \
  if ((st = dalloc(h, &(ptr), (n))) != RIHV_OK) return cleanup(st)
  AL(h->tw_x, nx);
  AL(h->tw_y, ny);
  AL(h->phase, h->nxy);
  AL(h->amp, h->nxy);
  AL(h->inter, h->nvox);
  AL(h->partial, h->nxy * kMaxGroups);
  AL(h->spec, h->nxy);
  AL(h->sx[0], h->nxy);
  AL(h->sx[1], h->nxy);
  AL(h->bhat, h->nxy);
  AL(h->holo, h->nxy);
  AL(h->x, h->nvox);
  AL(h->y, h->nvox);
  AL(h->v, h->nvox);
  for (int c = 0; c < 3; ++c) {
    AL(h->pa[c], h->nvox);
    AL(h->pb[c], h->nvox);
  }
  AL(h->sc, 1);
  AL(h->red.partials, 4 * kRedBlocks);
  h->fin_ctas = tv_final_ctas(nx, ny, nz, 8);   // the smallest z-chunk the tuner tries
  AL(h->fin_partials, h->fin_ctas);
  AL(h->red.tickets, 8);
  AL(h->det_err, 1);
  AL(h->coo_counts, static_cast<size_t>(nz) * coo_segments(nx, ny));
  AL(h->coo_seg_off, static_cast<size_t>(nz) * coo_segments(nx, ny));
  AL(h->coo_bad, 1);
  AL(h->tv_err, 1);
  AL(h->occ, h->nz + 1);
#undef AL
  if (cudaMemset(h->red.tickets, 0, 8 * sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(h->det_err, 0, sizeof(int)) != cudaSuccess ||
      cudaMemset(h->tv_err, 0, sizeof(int)) != cudaSuccess)
    return cleanup(fail(h, RIHV_ERR_CUDA, "memset failed"));
  for (int b = 0; b < 3; ++b)
    for (int c = 0; c < 3; ++c) {
      const int rows = b == 0 ? kTvBoxH1 : (b == 1 ? kTv2BoxH : kTv2BoxHF);
      const int cols = b == 0 ? kTvBoxW : kTv2BoxW;
      if (make_volume_tmap(&h->tm_pa[b][c], h->pa[c], nx, ny, nz, rows, cols) != cudaSuccess ||
          make_volume_tmap(&h->tm_pb[b][c], h->pb[c], nx, ny, nz, rows, cols) != cudaSuccess)
        return cleanup(fail(h, RIHV_ERR_CUDA, "tensor map encoding failed"));
    }

  // Twiddles exp(-2 pi i m / n) in FP64, rounded to float.
  auto twiddles = [](int n) {
    std::vector<float2> t(n);
    for (int m = 0; m < n; ++m) {
      const double a = -2.0 * M_PI * m / n;
      t[m] = make_float2(static_cast<float>(std::cos(a)), static_cast<float>(std::sin(a)));
    }
    return t;
  };
  std::vector<float2> twx = twiddles(nx), twy = twiddles(ny);

  // Phase table of the angular-spectrum transfer function, strip-major
  // [nx/W][ny][W]: phi0 = frac(z0 kappa), phid = frac(dz kappa) in units of
  // 2^-32 cycle; amp = 1 on the propagating band.
  std::vector<uint2> ph(h->nxy);
  std::vector<float> am(h->nxy);
  const double il2 = 1.0 / (wavelength * wavelength);
  for (int ky = 0; ky < ny; ++ky) {
    const double fy = fft_freq(ky, ny, pitch);
    for (int kx = 0; kx < nx; ++kx) {
      const double fx = fft_freq(kx, nx, pitch);
      const bool prop = wavelength * wavelength * (fx * fx + fy * fy) < 1.0;
      const double kappa = prop ? std::sqrt(il2 - fx * fx - fy * fy) : 0.0;
      const size_t idx = (static_cast<size_t>(kx / kStrip) * ny + ky) * kStrip + (kx % kStrip);
      ph[idx] = make_uint2(to_cycles32(frac(z0 * kappa)), to_cycles32(frac(dz * kappa)));
      am[idx] = prop ? 1.f : 0.f;
    }
  }
  if (cudaMemcpy(h->tw_x, twx.data(), nx * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(h->tw_y, twy.data(), ny * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(h->phase, ph.data(), h->nxy * sizeof(uint2), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(h->amp, am.data(), h->nxy * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
    return cleanup(fail(h, RIHV_ERR_CUDA, "upload of tables failed"));

  // Step size tau = 1 / L, L = 2 max_f sum_j |H_j(f)|^2 = 2 nz on any
  // propagating frequency (0 if none propagates).
  bool any_prop = false;
  for (float a : am) any_prop |= (a > 0.f);
  h->tau = any_prop ? 1.0 / (2.0 * nz) : 0.0;

  // Kernel smem limits
  if (rows_smem_bytes(nx, 4) > 227 * 1024 || cols_smem_bytes(COL_FWD_ZSUM, ny) > 227 * 1024)
    return cleanup(fail(h, RIHV_ERR_UNSUPPORTED_SIZE, "shared memory limit"));
  *out = h;
  return RIHV_OK;
}

rihv_status rihv_destroy(rihv_handle h) {
  if (!h) return RIHV_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  for (void* p : h->allocs) cudaFree(p);
  if (h->det.label) cudaFree(h->det.label);
  if (h->det.cid) cudaFree(h->det.cid);
  if (h->det.block_counts) cudaFree(h->det.block_counts);
  if (h->det.maxbits) cudaFree(h->det.maxbits);
  if (h->det.ncomp) cudaFree(h->det.ncomp);
  if (h->det.stats) cudaFree(h->det.stats);
  if (h->det.first) cudaFree(h->det.first);
  for (void* p : {static_cast<void*>(h->cdet.lin), static_cast<void*>(h->cdet.wgt),
                  static_cast<void*>(h->cdet.label), static_cast<void*>(h->cdet.cid),
                  static_cast<void*>(h->cdet.block_counts), static_cast<void*>(h->cdet.maxbits),
                  static_cast<void*>(h->cdet.nhits), static_cast<void*>(h->cdet.ncomp)})
    if (p) cudaFree(p);
  if (h->trace) cudaFree(h->trace);
  for (auto e : h->ev_pool) cudaEventDestroy(e);
  delete h;
  return RIHV_OK;
}

rihv_status rihv_set_stream(rihv_handle h, void* stream) {
  if (!h) return fail(nullptr, RIHV_ERR_INVALID_ARG, "null handle");
  const int sd = stream_device(stream);
  if (sd != kLegacyStream && sd != h->device)
    return fail(h, RIHV_ERR_INVALID_ARG, "the stream belongs to device %d, the handle to device %d",
                sd, h->device);
  h->stream = static_cast<cudaStream_t>(stream);
  return RIHV_OK;
}

rihv_status rihv_set_options(rihv_handle h, const rihv_options* o) {
  if (!h || !o) return fail(h, RIHV_ERR_INVALID_ARG, "null argument");
  if ((o->tv_dims != 2 && o->tv_dims != 3) || o->n_inner < 0 || o->check_every < 0 ||
      o->tol < 0 || o->f_star < 0 || (o->restart != 0 && o->restart != 1) ||
      (o->accelerate != 0 && o->accelerate != 1) ||
      (o->tv_steps_per_launch != 1 && o->tv_steps_per_launch != 2) ||
      (o->fuse_finalize != 0 && o->fuse_finalize != 1) ||
      (o->skip_empty_planes != 0 && o->skip_empty_planes != 1) ||
      (o->tv_zchunk != 0 && (o->tv_zchunk < std::min(8, h->nz) || o->tv_zchunk > kTvMaxChunk)) ||
      (o->fft_rows_per_cta != 0 && o->fft_rows_per_cta != 1 && o->fft_rows_per_cta != 2 &&
       o->fft_rows_per_cta != 4 && o->fft_rows_per_cta != 8) ||
      (o->fft_rows_per_cta != 0 && h->ny % o->fft_rows_per_cta != 0) ||
      (o->tv_fgp != 0 && o->tv_fgp != 1) || (o->solver != 0 && o->solver != 1) ||
      (o->tv_split != 0 && o->tv_split != 1))
    return fail(h, RIHV_ERR_INVALID_ARG, "invalid options");
  // scratch of the optional iterations is allocated here, not inside a solve
  // (which may be being captured into a graph)
  if (o->tv_fgp && !h->pc[0])
    for (int c = 0; c < 3; ++c) {
      CKS(dalloc(h, &h->pc[c], h->nvox));
      CKS(dalloc(h, &h->pd[c], h->nvox));
    }
  if (o->solver == 1 && !h->fasta_g[0]) {
    CKS(dalloc(h, &h->fasta_g[0], h->nvox));
    CKS(dalloc(h, &h->fasta_g[1], h->nvox));
    CKS(dalloc(h, &h->fasta_x, h->nvox));
    CKS(dalloc(h, &h->fasta_dots, 4));
  }
  h->opt = *o;
  return RIHV_OK;
}

rihv_status rihv_step_size(rihv_handle h, double* tau) {
  if (!h || !tau) return fail(h, RIHV_ERR_INVALID_ARG, "null argument");
  *tau = h->tau;
  return RIHV_OK;
}

rihv_status rihv_forward(rihv_handle h, const void* x, void* out) {
  if (!h) return fail(nullptr, RIHV_ERR_INVALID_ARG, "null handle");
  CKS(check_dev(h, x, "x"));
  CKS(check_dev(h, out, "out"));
  CKS(forward_spectrum(h, static_cast<const float2*>(x), nullptr, h->spec));
  StageScope sc(h, ST_FORWARD, 2);
  CK(launch_cols(COL_PLAIN_INV, col_args(h, h->spec, h->inter), 1, h->stream));
  RowArgs ra = row_args(h, h->inter, static_cast<float2*>(out), 1);
  ra.scale = static_cast<float>(1.0 / static_cast<double>(h->nxy));
  CK(launch_rows(1, ROW_IN_STRIP, ROW_OUT_C64, ROW_EPI_SCALE, ra, h->stream));
  return RIHV_OK;
}

rihv_status rihv_adjoint(rihv_handle h, const void* r, void* out) {
  if (!h) return fail(nullptr, RIHV_ERR_INVALID_ARG, "null handle");
  CKS(check_dev(h, r, "r"));
  CKS(check_dev(h, out, "out"));
  {
    StageScope sc(h, ST_ADJOINT, 2);
    CKS(fft2_plane(h, r, false, h->spec));
  }
  return adjoint_planes(h, h->spec, nullptr, static_cast<float2*>(out),
                        static_cast<float>(1.0 / static_cast<double>(h->nxy)), false);
}

rihv_status rihv_prox_fused_lasso(rihv_handle h, const void* v, float t_l1, float t_tv,
                                  int inner_iters, void* x_out) {
  if (!h) return fail(nullptr, RIHV_ERR_INVALID_ARG, "null handle");
  CKS(check_dev(h, v, "v"));
  CKS(check_dev(h, x_out, "x_out"));
  if (!(t_l1 >= 0.f) || !(t_tv >= 0.f) || inner_iters < 0 || !std::isfinite(t_l1) ||
      !std::isfinite(t_tv))
    return fail(h, RIHV_ERR_INVALID_ARG, "t_l1, t_tv must be finite and >= 0, inner_iters >= 0");
  if (v == x_out) return fail(h, RIHV_ERR_INVALID_ARG, "v and x_out must not alias");
  return prox_into(h, static_cast<const float2*>(v), t_l1, t_tv, inner_iters, FIN_PROX,
                   static_cast<float2*>(x_out));
}

rihv_status rihv_solve(rihv_handle h, const float* hologram, float lambda_l1, float lambda_tv,
                       int iters, const void* x0, void* x_out, double* trace, int* iters_done) {
  if (!h) return fail(nullptr, RIHV_ERR_INVALID_ARG, "null handle");
  if (!hologram || !x_out) return fail(h, RIHV_ERR_INVALID_ARG, "hologram and x_out are required");
  CKS(check_solve_args(h, lambda_l1, lambda_tv, iters));
  if (is_device_ptr(x_out) && !aligned16(x_out))
    return fail(h, RIHV_ERR_INVALID_ARG, "x_out is not 16-byte aligned");
  for (const void* p : {static_cast<const void*>(hologram), x0, static_cast<const void*>(x_out)}) {
    const int where = p ? pointer_device(p) : kNotDevicePtr;
    if (where >= 0 && where != h->device)
      return fail(h, RIHV_ERR_INVALID_ARG, "a buffer lives on device %d, the handle on device %d",
                  where, h->device);
  }
  const size_t vb = h->nvox * sizeof(float2);
  const int M = h->opt.check_every;
  CKS(ensure_trace(h, (M > 0) ? iters / M : 0));
  const bool stop_test = h->opt.f_star > 0.0 && M > 0;

  CKS(copy_in(h, h->holo, hologram, h->nxy * sizeof(float)));
  if (x0) CKS(copy_in(h, h->x, x0, vb));
  int done = 0;
  int check = 0;
  if (h->opt.solver == 1)
    CKS(solve_fasta(h, x0 != nullptr, lambda_l1, lambda_tv, iters, &check, &done));
  else
    CKS(enqueue_setup(h, x0 != nullptr));
  for (int k = 1; k <= iters && h->opt.solver == 0; ++k) {
    const int before = check;
    CKS(enqueue_iteration(h, k, lambda_l1, lambda_tv, &check));
    done = k;
    if (stop_test && check > before) {
      double f = 0;
      CK(cudaMemcpyAsync(&f, h->trace + before, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
      if (f <= h->opt.f_star * (1.0 + h->opt.tol)) break;
    }
  }
  if (pointer_device(x_out) == kNotDevicePtr) {
    // host output: its pages are touched once the iterations have run
    CK(cudaStreamSynchronize(h->stream));
    touch_host_pages(x_out, vb);
  }
  CK(cudaMemcpyAsync(x_out, h->x, vb, cudaMemcpyDefault, h->stream));
  if (trace && check > 0)
    CK(cudaMemcpyAsync(trace, h->trace, sizeof(double) * check, cudaMemcpyDefault, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (iters_done) *iters_done = done;
  return read_solve_errors(h);
}

rihv_status rihv_fasta_steps(rihv_handle h, double* taus, int capacity, int* n_steps,
                             int* backtracks) {
  if (!h || !n_steps || capacity < 0 || (capacity > 0 && !taus))
    return fail(h, RIHV_ERR_INVALID_ARG, "invalid arguments");
  const int n = static_cast<int>(h->fasta_taus.size());
  for (int i = 0; i < n && i < capacity; ++i) taus[i] = h->fasta_taus[i];
  *n_steps = n;
  if (backtracks) *backtracks = h->fasta_backtracks;
  return RIHV_OK;
}

rihv_status rihv_coo_compact(rihv_handle h, const void* x, long long* plane_offsets, int* rows,
                             int* cols, void* vals, long long capacity, long long* nnz) {
  if (!h) return fail(nullptr, RIHV_ERR_INVALID_ARG, "null handle");
  if (!x) x = h->x;   // the last solve's result
  CKS(check_dev(h, x, "x"));
  if (!plane_offsets || !nnz || capacity < 0 || (capacity > 0 && (!rows || !cols || !vals)))
    return fail(h, RIHV_ERR_INVALID_ARG, "invalid COO arguments");
  CKS(check_dev(h, plane_offsets, "plane_offsets"));
  const float2* xv = static_cast<const float2*>(x);
  CK(launch_coo_count(xv, h->nx, h->ny, h->nz, h->coo_counts, h->coo_seg_off, plane_offsets,
                      h->stream));
  long long total = 0;
  CK(cudaMemcpyAsync(&total, plane_offsets + h->nz, sizeof(long long), cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaStreamSynchronize(h->stream));
  *nnz = total;
  if (total > capacity)
    return fail(h, RIHV_ERR_INVALID_ARG, "COO capacity %lld < %lld non-zeros", capacity, total);
  if (total > 0) {
    CKS(check_dev(h, rows, "rows"));
    CKS(check_dev(h, cols, "cols"));
    CKS(check_dev(h, vals, "vals"));
    CK(launch_coo_write(xv, h->nx, h->ny, h->nz, h->coo_seg_off, rows, cols,
                        static_cast<float2*>(vals), h->stream));
  }
  CK(cudaStreamSynchronize(h->stream));
  return RIHV_OK;
}

rihv_status rihv_coo_expand(rihv_handle h, const long long* plane_offsets, const int* rows,
                            const int* cols, const void* vals, long long nnz, void* x_out) {
  if (!h) return fail(nullptr, RIHV_ERR_INVALID_ARG, "null handle");
  if (!plane_offsets || !x_out || nnz < 0 || (nnz > 0 && (!rows || !cols || !vals)))
    return fail(h, RIHV_ERR_INVALID_ARG, "invalid COO arguments");
  CKS(check_dev(h, plane_offsets, "plane_offsets"));
  CKS(check_dev(h, x_out, "x_out"));
  // offsets are checked on the host before any entry is touched
  std::vector<long long> off(static_cast<size_t>(h->nz) + 1);
  CK(cudaMemcpyAsync(off.data(), plane_offsets, off.size() * sizeof(long long),
                     cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (off[0] != 0 || off[h->nz] != nnz)
    return fail(h, RIHV_ERR_INVALID_ARG, "plane offsets must run from 0 to nnz");
  for (int k = 0; k < h->nz; ++k)
    if (off[k + 1] < off[k] || off[k + 1] - off[k] > static_cast<long long>(h->nxy))
      return fail(h, RIHV_ERR_INVALID_ARG, "plane offsets must be non-decreasing, <= nx*ny per plane");
  if (nnz > 0) {
    CKS(check_dev(h, rows, "rows"));
    CKS(check_dev(h, cols, "cols"));
    CKS(check_dev(h, vals, "vals"));
  }
  CK(cudaMemsetAsync(h->coo_bad, 0, sizeof(int), h->stream));
  CK(launch_coo_scatter(rows, cols, static_cast<const float2*>(vals), plane_offsets, h->nx, h->ny,
                        h->nz, static_cast<float2*>(x_out), h->coo_bad, h->stream));
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, h->coo_bad, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (bad) return fail(h, RIHV_ERR_INVALID_ARG, "COO entry outside the plane (skipped)");
  return RIHV_OK;
}

rihv_status rihv_detect(rihv_handle h, const void* x, float rel_thresh, int min_vox,
                        rihv_particle* out, int max_out, int* n_out) {
  if (!h) return fail(nullptr, RIHV_ERR_INVALID_ARG, "null handle");
  if (!x) x = h->x;   // the last solve's result
  CKS(check_dev(h, x, "x"));
  if (!n_out || (max_out > 0 && !out) || max_out < 0 || min_vox < 0 || !(rel_thresh >= 0.f) ||
      !std::isfinite(rel_thresh))
    return fail(h, RIHV_ERR_INVALID_ARG, "invalid detect arguments");
  if (h->nvox >= static_cast<size_t>(INT32_MAX))
    return fail(h, RIHV_ERR_UNSUPPORTED_SIZE, "volume too large for int32 labels");
  DetectWork& w = h->det;
  const size_t nb = (h->nvox + 1023) / 1024;
  if (!w.label) {
    if (cudaMalloc(&w.label, h->nvox * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&w.cid, h->nvox * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&w.block_counts, nb * sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc(&w.maxbits, sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc(&w.ncomp, sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, RIHV_ERR_OOM, "detection scratch allocation failed");
    }
  }
  StageScope scope(h, ST_DETECT, 8);
  int ncomp = 0;
  CK(detect_label(static_cast<const float2*>(x), h->nx, h->ny, h->nz, rel_thresh, w, h->det_err,
                  &ncomp, h->stream));
  CKS(ensure_stats(h, ncomp));
  if (ncomp > 0)
    CK(detect_stats(static_cast<const float2*>(x), h->nx, h->ny, h->nz, w, ncomp, h->stream));
  return emit_particles(h, ncomp, min_vox, out, max_out, n_out);
}

rihv_status rihv_detect_coo(rihv_handle h, const long long* plane_offsets, const int* rows,
                            const int* cols, const void* vals, long long nnz, float rel_thresh,
                            int min_vox, rihv_particle* out, int max_out, int* n_out) {
  if (!h) return fail(nullptr, RIHV_ERR_INVALID_ARG, "null handle");
  if (!plane_offsets || nnz < 0 || (nnz > 0 && (!rows || !cols || !vals)) || !n_out ||
      (max_out > 0 && !out) || max_out < 0 || min_vox < 0 || !(rel_thresh >= 0.f) ||
      !std::isfinite(rel_thresh))
    return fail(h, RIHV_ERR_INVALID_ARG, "invalid detect arguments");
  if (nnz >= static_cast<long long>(INT32_MAX))
    return fail(h, RIHV_ERR_UNSUPPORTED_SIZE, "more non-zeros than int32 list positions");
  CKS(check_dev(h, plane_offsets, "plane_offsets"));
  *n_out = 0;
  if (nnz == 0) return RIHV_OK;
  CKS(check_dev(h, rows, "rows"));
  CKS(check_dev(h, cols, "cols"));
  CKS(check_dev(h, vals, "vals"));
  // plane offsets are checked on the host before any entry is read
  std::vector<long long> off(static_cast<size_t>(h->nz) + 1);
  CK(cudaMemcpyAsync(off.data(), plane_offsets, off.size() * sizeof(long long),
                     cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (off[0] != 0 || off[h->nz] != nnz)
    return fail(h, RIHV_ERR_INVALID_ARG, "plane offsets must run from 0 to nnz");
  for (int k = 0; k < h->nz; ++k)
    if (off[k + 1] < off[k] || off[k + 1] - off[k] > static_cast<long long>(h->nxy))
      return fail(h, RIHV_ERR_INVALID_ARG, "plane offsets must be non-decreasing, <= nx*ny per plane");
  CooDetectWork& w = h->cdet;
  if (static_cast<size_t>(nnz) > w.capacity) {
    for (void* p : {static_cast<void*>(w.lin), static_cast<void*>(w.wgt),
                    static_cast<void*>(w.label), static_cast<void*>(w.cid),
                    static_cast<void*>(w.block_counts)})
      if (p) cudaFree(p);
    w.lin = nullptr; w.wgt = nullptr; w.label = nullptr; w.cid = nullptr; w.block_counts = nullptr;
    w.capacity = 0;
    const size_t cap = std::max<size_t>(static_cast<size_t>(nnz), 1 << 16);
    if (cudaMalloc(&w.lin, cap * sizeof(long long)) != cudaSuccess ||
        cudaMalloc(&w.wgt, cap * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&w.label, cap * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&w.cid, cap * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&w.block_counts, (cap / 1024 + 1) * sizeof(unsigned)) != cudaSuccess ||
        (!w.maxbits && cudaMalloc(&w.maxbits, sizeof(unsigned)) != cudaSuccess) ||
        (!w.nhits && cudaMalloc(&w.nhits, sizeof(int)) != cudaSuccess) ||
        (!w.ncomp && cudaMalloc(&w.ncomp, sizeof(int)) != cudaSuccess)) {
      cudaGetLastError();
      return fail(h, RIHV_ERR_OOM, "detection list allocation failed");
    }
    w.capacity = cap;
  }
  StageScope scope(h, ST_DETECT, 9);
  int m = 0, ncomp = 0;
  CK(detect_coo_hits(plane_offsets, rows, cols, static_cast<const float2*>(vals), nnz, h->nx,
                     h->ny, h->nz, rel_thresh, w, &m, h->stream));
  if (m > 0)
    CK(detect_coo_label(m, h->nx, h->ny, w, h->det_err, &ncomp, h->stream));
  CKS(ensure_stats(h, ncomp));
  if (ncomp > 0)
    CK(detect_coo_stats(m, h->nx, h->ny, w, ncomp, h->det.stats, h->det.first, h->stream));
  return emit_particles(h, ncomp, min_vox, out, max_out, n_out);
}

rihv_status rihv_selftest_bounded_wait(rihv_handle h, int polls) {
  if (!h) return fail(nullptr, RIHV_ERR_INVALID_ARG, "null handle");
  if (polls < 1 || polls > (1 << 22))
    return fail(h, RIHV_ERR_INVALID_ARG, "polls must be in [1, 2^22]");
  int flag = 0;
  CK(cudaMemsetAsync(h->tv_err, 0, sizeof(int), h->stream));
  CK(launch_wait_selftest(h->tv_err, polls, h->stream));
  CK(cudaMemcpyAsync(&flag, h->tv_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaMemsetAsync(h->tv_err, 0, sizeof(int), h->stream));
  if (flag) return fail(h, RIHV_ERR_TIMEOUT, "bounded wait gave up after %d polls (self-test)", polls);
  return fail(h, RIHV_ERR_CUDA, "self-test barrier completed although nothing arrived on it");
}

rihv_status rihv_set_profiling(rihv_handle h, int on) {
  if (!h) return fail(nullptr, RIHV_ERR_INVALID_ARG, "null handle");
  if (on && h->ev_pool.empty()) {
    h->ev_pool.resize(kEventPool);
    for (auto& e : h->ev_pool) CK(cudaEventCreate(&e));
  }
  h->prof = on < 0 ? 0 : (on > 2 ? 2 : on);
  return RIHV_OK;
}

rihv_status rihv_stage_times(rihv_handle h, double* ms, long long* launches, int n) {
  if (!h) return fail(nullptr, RIHV_ERR_INVALID_ARG, "null handle");
  CK(cudaStreamSynchronize(h->stream));
  for (auto& r : h->recs) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, r.a, r.b));
    h->stage_ms[r.stage] += t;
  }
  h->recs.clear();
  h->ev_used = 0;
  for (int i = 0; i < kNumStages && i < n; ++i) {
    if (ms) ms[i] = h->stage_ms[i];
    if (launches) launches[i] = h->stage_launches[i];
    h->stage_ms[i] = 0;
    h->stage_launches[i] = 0;
  }
  return RIHV_OK;
}

// -----------------------------------------------------------------------------
// Batched solves (one CUDA graph per batch)
// -----------------------------------------------------------------------------
rihv_status rihv_batch_create(const rihv_handle* hs, int n, rihv_batch* out) {
  if (!hs || n <= 0 || !out) return fail(nullptr, RIHV_ERR_INVALID_ARG, "invalid batch arguments");
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!hs[i]) return fail(nullptr, RIHV_ERR_INVALID_ARG, "null handle in batch");
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return fail(nullptr, RIHV_ERR_INVALID_ARG, "a handle appears twice");
  }
  rihv_batch b = new (std::nothrow) rihv_batch_st();
  if (!b) return fail(nullptr, RIHV_ERR_OOM, "host allocation failed");
  b->hs.assign(hs, hs + n);
  bool ok = cudaStreamCreateWithFlags(&b->master, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
  b->branch.resize(n, nullptr);
  b->join.resize(n, nullptr);
  for (int i = 0; ok && i < n; ++i)
    ok = cudaStreamCreateWithFlags(&b->branch[i], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaMalloc(&b->done_dev, sizeof(int) * n) == cudaSuccess;
  b->done.assign(n, 0);
  if (!ok) {
    rihv_batch_destroy(b);
    return fail(nullptr, RIHV_ERR_CUDA, "stream, event or counter allocation failed");
  }
  *out = b;
  return RIHV_OK;
}

rihv_status rihv_batch_destroy(rihv_batch b) {
  if (!b) return RIHV_OK;
  if (b->master) cudaStreamSynchronize(b->master);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (auto s : b->branch)
    if (s) cudaStreamDestroy(s);
  for (auto e : b->join)
    if (e) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->master) cudaStreamDestroy(b->master);
  if (b->done_dev) cudaFree(b->done_dev);
  delete b;
  return RIHV_OK;
}

static bool same_options(const rihv_options& a, const rihv_options& o) {
  return a.tv_dims == o.tv_dims && a.restart == o.restart && a.accelerate == o.accelerate &&
         a.n_inner == o.n_inner && a.check_every == o.check_every &&
         a.tv_steps_per_launch == o.tv_steps_per_launch && a.fuse_finalize == o.fuse_finalize &&
         a.f_star == o.f_star && a.tol == o.tol && a.skip_empty_planes == o.skip_empty_planes &&
         a.tv_zchunk == o.tv_zchunk && a.fft_rows_per_cta == o.fft_rows_per_cta &&
         a.tv_fgp == o.tv_fgp && a.solver == o.solver && a.tv_split == o.tv_split;
}

// Captures `fn` (enqueueing on h's stream, switched to `st` meanwhile) into a
// standalone graph.
static rihv_status capture_graph(rihv_ctx* h, cudaStream_t st, cudaGraph_t* g,
                                 const std::function<rihv_status()>& fn) {
  cudaStream_t saved = h->stream;
  const int saved_prof = h->prof;
  h->stream = st;
  h->prof = 0;
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    h->stream = saved;
    h->prof = saved_prof;
    return fail(h, RIHV_ERR_CUDA, "begin capture: %s", cudaGetErrorString(e));
  }
  rihv_status r = fn();
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(st, &graph);
  h->stream = saved;
  h->prof = saved_prof;
  if (r != RIHV_OK) {
    if (graph) cudaGraphDestroy(graph);
    return r;
  }
  if (e != cudaSuccess) return fail(h, RIHV_ERR_CUDA, "end capture: %s", cudaGetErrorString(e));
  *g = graph;
  return RIHV_OK;
}

// Batched graph with a stop test per hologram (handles with f_star > 0):
// setup, then the iterations in chunks of check_every, each chunk after the
// first inside an IF node whose condition the previous chunk's last kernel
// sets from its objective (stop once F(x_k) <= f_star (1 + tol)). So every
// hologram stops at the first check that meets its
// tolerance, exactly where rihv_solve would, while the batch shares one graph.
// Handles without a stop test run all iterations in one child graph.
static rihv_status batch_capture_cond(rihv_batch b, float l1, float ltv, int iters, bool warm) {
  const int n = static_cast<int>(b->hs.size());
  rihv_ctx* h0 = b->hs[0];
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  b->launches.assign(n, std::vector<long long>(kNumStages, 0));
  b->checks.assign(n, 0);
  cudaGraph_t root = nullptr;
  if (cudaGraphCreate(&root, 0) != cudaSuccess) return fail(h0, RIHV_ERR_CUDA, "graph create");
  std::vector<cudaGraph_t> parts;   // standalone graphs, destroyed after cloning
  auto add_child = [&](cudaGraph_t into, cudaGraph_t g, const cudaGraphNode_t* dep,
                       cudaGraphNode_t* node) {
    parts.push_back(g);
    return cudaGraphAddChildGraphNode(node, into, dep, dep ? 1 : 0, g);
  };
  rihv_status st = RIHV_OK;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < n && st == RIHV_OK && e == cudaSuccess; ++i) {
    rihv_ctx* h = b->hs[i];
    const int M = h->opt.check_every;
    const bool stop = h->opt.f_star > 0.0 && M > 0;
    const double thr = h->opt.f_star * (1.0 + h->opt.tol);
    long long before[kNumStages];
    for (int s = 0; s < kNumStages; ++s) before[s] = h->stage_launches[s];
    cudaGraph_t g = nullptr;
    cudaGraphNode_t prev = nullptr, node = nullptr;
    int check = 0;
    h->batch_chunks = n > 1;   // a batch of one runs like a lone solve
    st = capture_graph(h, b->branch[i], &g, [&] { return enqueue_setup(h, warm); });
    if (st != RIHV_OK) {
      h->batch_chunks = false;
      break;
    }
    e = add_child(root, g, nullptr, &node);
    prev = node;
    const int chunk = stop ? M : iters;
    cudaGraphConditionalHandle next = 0;
    for (int k0 = 1; k0 <= iters && st == RIHV_OK && e == cudaSuccess; k0 += chunk) {
      const int k1 = std::min(iters, k0 + chunk - 1);
      const bool has_next = stop && k1 < iters && k1 % M == 0;
      cudaGraphConditionalHandle mine = next;
      next = 0;
      if (has_next) {
        e = cudaGraphConditionalHandleCreate(&next, root, 0, cudaGraphCondAssignDefault);
        if (e != cudaSuccess) break;
      }
      const double* fk = nullptr;
      st = capture_graph(h, b->branch[i], &g, [&]() -> rihv_status {
        for (int k = k0; k <= k1; ++k) CKS(enqueue_iteration(h, k, l1, ltv, &check));
        fk = (M > 0 && k1 % M == 0 && check > 0) ? h->trace + (check - 1) : nullptr;
        CK(launch_chunk_end(b->done_dev + i, k1, fk, thr, next, has_next ? 1 : 0, h->stream));
        return RIHV_OK;
      });
      if (st != RIHV_OK) break;
      if (k0 == 1) {
        e = add_child(root, g, &prev, &node);
      } else {
        // IF node on the condition the previous chunk set
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = mine;
        cp.conditional.type = cudaGraphCondTypeIf;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&node, root, &prev, nullptr, 1, &cp);
        if (e == cudaSuccess) {
          cudaGraphNode_t inner = nullptr;
          e = add_child(cp.conditional.phGraph_out[0], g, nullptr, &inner);
        }
      }
      prev = node;
    }
    h->batch_chunks = false;
    b->checks[i] = check;
    for (int s = 0; s < kNumStages; ++s) {
      b->launches[i][s] = h->stage_launches[s] - before[s];
      h->stage_launches[s] = before[s];   // counted per graph launch instead (upper bound)
    }
  }
  for (auto g : parts) cudaGraphDestroy(g);
  if (st == RIHV_OK && e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, root, 0);
  cudaGraphDestroy(root);
  if (st != RIHV_OK) return st;
  if (e != cudaSuccess) {
    b->exec = nullptr;
    return fail(h0, RIHV_ERR_CUDA, "conditional batch graph: %s", cudaGetErrorString(e));
  }
  b->conditional = true;
  b->iters = iters;
  b->l1 = l1;
  b->ltv = ltv;
  b->warm = warm;
  b->opts.clear();
  b->tunes.clear();
  for (auto* h : b->hs) {
    b->opts.push_back(h->opt);
    b->tunes.push_back(h->tv_zchunk);
    b->tunes.push_back(h->zpg);
    b->tunes.push_back(h->row_teams);
  }
  return RIHV_OK;
}

static rihv_status batch_capture(rihv_batch b, float l1, float ltv, int iters, bool warm) {
  const int n = static_cast<int>(b->hs.size());
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  std::vector<cudaStream_t> saved(n);
  std::vector<int> saved_prof(n);
  b->launches.assign(n, std::vector<long long>(kNumStages, 0));
  b->checks.assign(n, 0);
  rihv_ctx* h0 = b->hs[0];
  cudaError_t e = cudaStreamBeginCapture(b->master, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return fail(h0, RIHV_ERR_CUDA, "begin capture: %s", cudaGetErrorString(e));
  cudaEventRecord(b->fork, b->master);
  rihv_status st = RIHV_OK;
  for (int i = 0; i < n && st == RIHV_OK; ++i) {
    rihv_ctx* h = b->hs[i];
    saved[i] = h->stream;
    saved_prof[i] = h->prof;
    h->stream = b->branch[i];
    h->prof = 0;
    long long before[kNumStages];
    for (int s = 0; s < kNumStages; ++s) before[s] = h->stage_launches[s];
    cudaStreamWaitEvent(b->branch[i], b->fork, 0);
    h->batch_chunks = n > 1;   // a batch of one runs like a lone solve
    st = enqueue_setup(h, warm);
    int check = 0;
    for (int k = 1; k <= iters && st == RIHV_OK; ++k) st = enqueue_iteration(h, k, l1, ltv, &check);
    h->batch_chunks = false;
    b->checks[i] = check;
    for (int s = 0; s < kNumStages; ++s) {
      b->launches[i][s] = h->stage_launches[s] - before[s];
      h->stage_launches[s] = before[s];   // counted per graph launch instead
    }
    cudaEventRecord(b->join[i], b->branch[i]);
    cudaStreamWaitEvent(b->master, b->join[i], 0);
  }
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(b->master, &graph);
  for (int i = 0; i < n; ++i) {
    if (!saved.empty() && i < static_cast<int>(saved.size()) && b->hs[i]->stream == b->branch[i]) {
      b->hs[i]->stream = saved[i];
      b->hs[i]->prof = saved_prof[i];
    }
  }
  if (st != RIHV_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return fail(h0, RIHV_ERR_CUDA, "end capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&b->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    b->exec = nullptr;
    return fail(h0, RIHV_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  b->conditional = false;
  b->iters = iters;
  b->l1 = l1;
  b->ltv = ltv;
  b->warm = warm;
  b->opts.clear();
  b->tunes.clear();
  for (auto* h : b->hs) {
    b->opts.push_back(h->opt);
    b->tunes.push_back(h->tv_zchunk);
    b->tunes.push_back(h->zpg);
    b->tunes.push_back(h->row_teams);
  }
  return RIHV_OK;
}

rihv_status rihv_batch_solve(rihv_batch b, const float* const* holograms, float lambda_l1,
                             float lambda_tv, int iters, const void* const* x0s, void* const* x_outs,
                             double* const* traces) {
  if (!b) return fail(nullptr, RIHV_ERR_INVALID_ARG, "null batch");
  const int n = static_cast<int>(b->hs.size());
  rihv_ctx* h0 = b->hs[0];
  if (!holograms || !x_outs) return fail(h0, RIHV_ERR_INVALID_ARG, "holograms and x_outs required");
  for (int i = 0; i < n; ++i) {
    rihv_ctx* h = b->hs[i];
    if (!holograms[i] || !x_outs[i]) return fail(h, RIHV_ERR_INVALID_ARG, "null hologram or x_out");
    CKS(check_solve_args(h, lambda_l1, lambda_tv, iters));
    const int M = h->opt.check_every;
    CKS(ensure_trace(h, (M > 0) ? iters / M : 0));
  }
  for (auto* h : b->hs)
    if (h->opt.solver != 0)
      return fail(h, RIHV_ERR_INVALID_ARG, "the FASTA solver decides its steps on the host; "
                                          "batched graphs run FISTA only");
  bool cond = false;   // some hologram has a stop test: graph with IF nodes
  for (auto* h : b->hs) cond = cond || (h->opt.f_star > 0.0 && h->opt.check_every > 0);
  const bool warm = x0s != nullptr;
  bool recapture = !b->exec || b->iters != iters || b->l1 != lambda_l1 || b->ltv != lambda_tv ||
                   b->warm != warm || b->conditional != cond;
  for (int i = 0; i < n && !recapture; ++i) {
    rihv_ctx* h = b->hs[i];
    recapture = !same_options(b->opts[i], h->opt) || b->tunes[3 * i] != h->tv_zchunk ||
                b->tunes[3 * i + 1] != h->zpg || b->tunes[3 * i + 2] != h->row_teams;
  }
  // inputs into each handle's own buffers (outside the graph)
  for (int i = 0; i < n; ++i) {
    rihv_ctx* h = b->hs[i];
    touch_host_pages(holograms[i], h->nxy * sizeof(float));
    CK(cudaMemcpyAsync(h->holo, holograms[i], h->nxy * sizeof(float), cudaMemcpyDefault, b->master));
    if (warm) {
      if (!x0s[i]) return fail(h, RIHV_ERR_INVALID_ARG, "x0s given but x0s[i] is NULL");
      touch_host_pages(x0s[i], h->nvox * sizeof(float2));
      CK(cudaMemcpyAsync(h->x, x0s[i], h->nvox * sizeof(float2), cudaMemcpyDefault, b->master));
    }
  }
  if (recapture)
    CKS(cond ? batch_capture_cond(b, lambda_l1, lambda_tv, iters, warm)
             : batch_capture(b, lambda_l1, lambda_tv, iters, warm));
  rihv_ctx* h = h0;
  if (cond) {   // objective checks a hologram does not reach read as NaN
    for (int i = 0; i < n; ++i)
      if (b->checks[i] > 0)
        CK(cudaMemsetAsync(b->hs[i]->trace, 0xFF, sizeof(double) * b->checks[i], b->master));
  }
  CK(cudaGraphLaunch(b->exec, b->master));
  bool host_out = false;   // host outputs: their pages are touched once the graph has run
  for (int i = 0; i < n; ++i) host_out = host_out || pointer_device(x_outs[i]) == kNotDevicePtr;
  if (host_out) {
    CK(cudaStreamSynchronize(b->master));
    for (int i = 0; i < n; ++i) touch_host_pages(x_outs[i], b->hs[i]->nvox * sizeof(float2));
  }
  for (int i = 0; i < n; ++i) {
    rihv_ctx* hi = b->hs[i];
    for (int s = 0; s < kNumStages; ++s) hi->stage_launches[s] += b->launches[i][s];
    CK(cudaMemcpyAsync(x_outs[i], hi->x, hi->nvox * sizeof(float2), cudaMemcpyDefault, b->master));
    if (traces && traces[i] && b->checks[i] > 0)
      CK(cudaMemcpyAsync(traces[i], hi->trace, sizeof(double) * b->checks[i], cudaMemcpyDefault,
                         b->master));
  }
  if (cond)
    CK(cudaMemcpyAsync(b->done.data(), b->done_dev, sizeof(int) * n, cudaMemcpyDeviceToHost,
                       b->master));
  CK(cudaStreamSynchronize(b->master));
  if (!cond) std::fill(b->done.begin(), b->done.end(), iters);
  for (auto* hi : b->hs) CKS(read_solve_errors(hi));
  return RIHV_OK;
}

rihv_status rihv_batch_iterations(rihv_batch b, int* iters_done) {
  if (!b || !iters_done) return fail(nullptr, RIHV_ERR_INVALID_ARG, "null argument");
  for (size_t i = 0; i < b->done.size(); ++i) iters_done[i] = b->done[i];
  return RIHV_OK;
}

// -----------------------------------------------------------------------------
// Autotuner
// -----------------------------------------------------------------------------
static double time_ms(rihv_ctx* h, const std::function<rihv_status()>& fn, int reps,
                      rihv_status* st) {
  cudaEvent_t a, c;
  cudaEventCreate(&a);
  cudaEventCreate(&c);
  *st = fn();   // warm-up
  std::vector<float> t;
  for (int r = 0; r < reps && *st == RIHV_OK; ++r) {
    cudaEventRecord(a, h->stream);
    *st = fn();
    cudaEventRecord(c, h->stream);
    cudaEventSynchronize(c);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, c);
    t.push_back(ms);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(c);
  if (t.empty()) return 1e30;
  std::sort(t.begin(), t.end());
  return t[t.size() / 2];
}

rihv_status rihv_tv_split_plan(int nx, int ny, int nz, int final, int zchunk, int sms, int* out2) {
  if (nx <= 0 || ny <= 0 || nz <= 0 || zchunk <= 0 || sms <= 0 || !out2 || (final != 0 && final != 1))
    return fail(nullptr, RIHV_ERR_INVALID_ARG, "invalid arguments");
  const int tx = final ? kTv2TxF : kTv2Tx, ty = final ? kTv2TyF : kTv2Ty;
  const int ntiles = ((nx + tx - 1) / tx) * ((ny + ty - 1) / ty);
  tv_choose_split(ntiles, nz, std::min(zchunk, nz), final ? 4 : 3, sms, &out2[0], &out2[1]);
  return RIHV_OK;
}

rihv_status rihv_tv_schedule(rihv_handle h, int final, int* out3) {
  if (!h || !out3 || (final != 0 && final != 1)) return fail(h, RIHV_ERR_INVALID_ARG, "invalid arguments");
  const int zc = tv_launch_zchunk(h, 2, 2, final != 0);
  int split = 0, zc2 = 0;
  if (h->opt.tv_split) tv_split_for(h, final != 0, zc, &split, &zc2);
  out3[0] = zc;
  out3[1] = split;
  out3[2] = zc2;
  return RIHV_OK;
}

rihv_status rihv_autotune(rihv_handle h, const char* cache_path, int* chosen) {
  if (!h) return fail(nullptr, RIHV_ERR_INVALID_ARG, "null handle");
  char key[96];
  snprintf(key, sizeof(key), "rihv-tune-v2 %d %d %d %d", h->nx, h->ny, h->nz, h->opt.tv_dims);
  int zchunk = -1, per = -1, zpg = -1, teams = -1;
  if (cache_path) {
    if (FILE* f = fopen(cache_path, "r")) {
      char line[256];
      while (fgets(line, sizeof(line), f)) {
        int a = 0, b2 = 0, c = 0, d = 0;
        const size_t kl = strlen(key);
        if (strncmp(line, key, kl) == 0 && line[kl] == ':' &&
            sscanf(line + kl + 1, "%d %d %d %d", &a, &b2, &c, &d) == 4 && a >= 1 &&
            (b2 == 1 || b2 == 2) && c >= 1 && c <= h->nz && (h->nz + c - 1) / c <= kMaxGroups &&
            (d == 2 || d == 4 || d == 8) && h->ny % d == 0) {
          zchunk = a;
          per = b2;
          zpg = c;
          teams = d;
        }
      }
      fclose(f);
    }
  }
  if (zchunk < 0) {
    // Search on the handle's own buffers (values do not change the timing).
    CK(cudaMemsetAsync(h->v, 0, h->nvox * sizeof(float2), h->stream));
    CK(cudaMemsetAsync(h->y, 0, h->nvox * sizeof(float2), h->stream));
    CK(cudaMemsetAsync(h->spec, 0, h->nxy * sizeof(float2), h->stream));
    const int prof = h->prof;
    h->prof = 0;
    const rihv_options saved = h->opt;
    h->opt.tv_zchunk = 0;          // explicit choices would override the candidates
    h->opt.fft_rows_per_cta = 0;
    h->opt.tv_fgp = 0;
    const int saved_zc = h->tv_zchunk, saved_zpg = h->zpg, saved_g = h->groups;
    const int saved_teams = h->row_teams;
    rihv_status st = RIHV_OK;
    double best = 1e30;
    const int kSteps = 4;
    // candidates: powers of two, and for two steps per launch also the
    // default chunk
    const int zc_def = tv_default_zchunk(h->nx, h->ny, h->nz, 2, h->sms);
    for (int p = 2; p >= 1; --p) {
      // the default (two steps, the wave-filling chunk) first: another
      // candidate must beat it by 1 %
      std::vector<int> zcs = {8, 16, 32, 64, 128, 256};
      if (p == 2) {
        zcs.erase(std::remove(zcs.begin(), zcs.end(), zc_def), zcs.end());
        zcs.insert(zcs.begin(), zc_def);
      }
      for (int zc : zcs) {
        if (zc > h->nz && zc != 8) continue;
        h->opt.tv_steps_per_launch = p;
        h->tv_zchunk = zc;
        float2* const* pf = nullptr;
        const double t = time_ms(h, [&] { return tv_steps(h, h->v, 1e-3f, kSteps, &pf); }, 3, &st);
        if (st != RIHV_OK) break;
        if (t < best * 0.99) {
          best = t;
          zchunk = zc;
          per = p;
        }
      }
    }
    // column-pass z-groups: the wave-filling default and its neighbours
    best = 1e30;
    std::vector<int> cands;
    for (int g : {saved_g - 2, saved_g - 1, saved_g, saved_g + 1, saved_g + 2, 2 * saved_g}) {
      if (g < 1 || g > kMaxGroups || g > h->nz) continue;
      const int c = (h->nz + g - 1) / g;
      if (std::find(cands.begin(), cands.end(), c) == cands.end()) cands.push_back(c);
    }
    const float gs = static_cast<float>(2.0 * h->tau / static_cast<double>(h->nxy));
    for (int c : cands) {
      if (st != RIHV_OK) break;
      h->zpg = c;
      h->groups = (h->nz + c - 1) / c;
      const double t = time_ms(h, [&] {
        rihv_status s2 = forward_spectrum(h, h->y, nullptr, h->spec);
        if (s2 != RIHV_OK) return s2;
        return adjoint_planes(h, h->spec, h->y, h->v, gs, true);
      }, 3, &st);
      if (t < best * 0.99) {
        best = t;
        zpg = c;
      }
    }
    // row-pass tile: transforms per CTA of the register engine (1, 2, 4 or
    // 8 rows), with the chosen column z-groups
    const int teams0 = default_row_teams(h->nx, h->ny);
    teams = teams0;
    if (reg_length(h->nx) && st == RIHV_OK) {
      h->zpg = zpg;
      h->groups = (h->nz + zpg - 1) / zpg;
      best = 1e30;
      for (int t : kRowTeams) {
        if (h->ny % t != 0 || rows_smem_bytes(h->nx, t) > 227 * 1024) continue;
        h->row_teams = t;
        const double ms = time_ms(h, [&] {
          rihv_status s2 = forward_spectrum(h, h->y, nullptr, h->spec);
          if (s2 != RIHV_OK) return s2;
          return adjoint_planes(h, h->spec, h->y, h->v, gs, true);
        }, 3, &st);
        if (st != RIHV_OK) break;
        // the default unless clearly slower
        if (ms < best * 0.99 || (t == teams0 && ms < best * 1.01)) {
          best = ms;
          teams = t;
        }
      }
    }
    h->opt = saved;
    h->tv_zchunk = saved_zc;
    h->zpg = saved_zpg;
    h->groups = saved_g;
    h->row_teams = saved_teams;
    h->prof = prof;
    // reset the launch counters the search added
    for (int s = 0; s < kNumStages; ++s) h->stage_launches[s] = 0;
    if (st != RIHV_OK) return st;
    if (cache_path) {
      if (FILE* f = fopen(cache_path, "a")) {
        fprintf(f, "%s: %d %d %d %d\n", key, zchunk, per, zpg, teams);
        fclose(f);
      }
    }
  }
  h->tv_zchunk = zchunk;
  h->opt.tv_steps_per_launch = per;
  h->zpg = zpg;
  h->groups = (h->nz + zpg - 1) / zpg;
  h->row_teams = teams;
  if (chosen) {
    chosen[0] = zchunk;
    chosen[1] = per;
    chosen[2] = zpg;
    chosen[3] = teams;
  }
  return RIHV_OK;
}

}  // extern "C"

