/*
 * rihv.h - C ABI of the GB300 fused-lasso holographic volume reconstruction
 * library (librihv.so).
 *
 * Method: "Regularized Inverse Holographic Volume Reconstruction for 3D
 * Particle Tracking" (arXiv 1904.04884), Section 2. The library recovers a
 * complex volume x [nz][ny][nx] from one real hologram b [ny][nx] by solving
 *     min_x ||H x - b||_2^2 + lambda_l1 ||x||_1 + lambda_tv ||x||_TV
 * with FISTA, where H is the linearised angular-spectrum forward model.
 *
 * Conventions shared by every entry point
 *  - Volumes are complex64 (interleaved re, im float32), C order [nz][ny][nx],
 *    x fastest. Holograms are float32 [ny][nx]. Spectral/2D fields are
 *    complex64 [ny][nx].
 *  - Plane j lies at depth z_j = z0 + j*dz. Frequencies are in FFT order,
 *    f_x = k_x / (nx * pitch). The transfer function of plane j is
 *    H_j(f) = exp(i 2 pi z_j sqrt(1/wavelength^2 - f_x^2 - f_y^2)) on the
 *    propagating band and 0 for evanescent frequencies; it is generated inside
 *    the kernels, never stored.
 *  - Supported sizes: nx, ny in {n = 2^a * 3^b : 16 <= n <= 1024, a >= 3,
 *    b <= 1}; 1 <= nz <= 4096. Other sizes return RIHV_ERR_UNSUPPORTED_SIZE.
 *  - Pointers marked "device" must be CUDA device memory of the current
 *    device, 16-byte aligned and not overlapping each other. Pointers marked
 *    "host or device" may also be host memory (pinned or pageable); the
 *    library copies it with cudaMemcpyAsync on the handle's stream into or
 *    out of its own device buffers, and the call synchronises the stream.
 *  - All work is queued on the handle's stream (rihv_set_stream; default: the
 *    legacy default stream). Calls return once the work is queued unless they
 *    say otherwise. The caller owns every pointer it passes; the library owns
 *    its scratch, which rihv_create allocates and rihv_destroy frees. Only
 *    rihv_create, rihv_detect (labelling scratch) and rihv_solve (a larger
 *    objective trace than before) allocate; the iteration itself never does.
 *  - Errors: every call returns a status; arguments are checked before any
 *    launch. rihv_last_error() gives a message for the last failing call on
 *    the handle. A handle is not thread safe.
 */
#ifndef RIHV_H
#define RIHV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rihv_ctx* rihv_handle;

typedef enum {
  RIHV_OK = 0,
  RIHV_ERR_INVALID_ARG = 1,      /* bad pointer, size, alignment or value    */
  RIHV_ERR_CUDA = 2,             /* a CUDA runtime call failed               */
  RIHV_ERR_OOM = 3,              /* device allocation failed                 */
  RIHV_ERR_NONFINITE = 4,        /* objective or a norm became NaN/Inf       */
  RIHV_ERR_TIMEOUT = 5,          /* a bounded device wait gave up            */
  RIHV_ERR_UNSUPPORTED_SIZE = 6  /* grid size outside the supported set      */
} rihv_status;

/* Solver options. Defaults (rihv_default_options): tv_dims 3, restart 1,
 * accelerate 1, n_inner 20, check_every 10, tol 0, f_star 0,
 * tv_steps_per_launch 2, fuse_finalize 1, skip_empty_planes 0, tv_zchunk 0,
 * fft_rows_per_cta 0, tv_fgp 0, solver 0, tv_split 1. */
typedef struct {
  int tv_dims;       /* 3: 3D isotropic TV; 2: plane-wise 2D TV (Section 2,
                        TV prox paragraph restricts TV to planes)            */
  int restart;       /* 1: gradient restart (O'Donoghue-Candes) on           */
  int accelerate;    /* 1: FISTA momentum; 0: ISTA (t == 1)                  */
  int n_inner;       /* TV dual gradient-projection steps per prox (>= 0)    */
  int check_every;   /* evaluate F(x_k) every M iterations (0: never)        */
  double tol;        /* with f_star > 0: stop at the first check where       */
  double f_star;     /*   F(x_k) <= f_star * (1 + tol)                       */
  int tv_steps_per_launch; /* 1: one dual step per kernel launch; 2: two
                        steps per launch (same arithmetic, the first step
                        recomputed on a one-voxel halo ring; an odd step
                        count starts with a one-step launch). 2 needs nx
                        even, which every supported size is.                 */
  int fuse_finalize; /* 1: with two steps per launch and >= 2 steps, the
                        last TV launch also forms x = soft(v - mu D^H p)
                        (and FISTA's y and restart product), so the final
                        dual never reaches memory; 0: separate finalize
                        kernel. Same arithmetic either way.                  */
  int skip_empty_planes; /* 1: the fused finalize records which planes of
                        x_k and y_{k+1} hold a non-zero voxel, and the next
                        forward propagations (of y_{k+1}, and of x_k for the
                        objective) skip the 2D FFTs and z-sum terms of the
                        all-zero planes (Section 2: the volume is sparse and
                        each plane propagates independently). Exact: a zero
                        plane adds nothing to the sum. Off by default: the
                        recording costs the finalize launch a few per cent
                        and pays only where solutions leave whole planes
                        empty. Takes effect when the finalize is fused
                        (fuse_finalize 1, two steps per launch, n_inner >= 2,
                        lambda_tv > 0) and nx, ny <= 1024; otherwise every
                        plane is propagated.                                 */
  int tv_zchunk;     /* planes per z-chunk of every TV launch (a CTA marches
                        its tile through one chunk): 0 (default) picks the
                        chunk per launch kind from the grid and the SM count
                        (or the autotuner's choice); otherwise
                        min(nz, 8) <= tv_zchunk <= 256, capped at nz. Results
                        do not depend on it, except the FISTA restart
                        product's summation order in the fused finalize.    */
  int fft_rows_per_cta; /* rows transformed per CTA in the row passes of the
                        register FFT engine (power-of-two nx): 0 (default)
                        takes the autotuner's choice, else 2 for nx >= 512
                        and 4 below; otherwise 1, 2, 4 or 8, dividing ny.
                        Same arithmetic for every value.                    */
  int tv_fgp;        /* 1: the TV prox runs the accelerated dual iteration
                        (Beck-Teboulle's fast gradient projection: each step
                        taken at r_k = p_{k-1} + ((t_{k-1} - 1)/t_k)(p_{k-1} -
                        p_{k-2})), one step per launch, separate finalize;
                        the first use allocates three more dual volumes'
                        worth of scratch (6 x 8 B per voxel). 0 (default):
                        gradient projection (Section 2, TV prox paragraph).  */
  int solver;        /* 0 (default): FISTA with gradient restart (Section 2,
                        FISTA paragraph). 1: forward-backward splitting with
                        FASTA's adaptive spectral step and non-monotone
                        backtracking (window 10, step halved on a failed
                        test, at most 20 times; first step 1/L); its host
                        loop synchronises twice per iteration, and the first
                        use allocates two gradient volumes and a candidate.  */
  int tv_split;      /* 1 (default): two-step TV launches whose equal z-chunks
                        would leave the last wave of CTAs partly idle cut the
                        last tiles into 2-4 shorter z-chunks, launched after
                        the rest (chosen by a makespan model of the launch,
                        taken when it saves at least 2 %); 0: equal z-chunks
                        for every tile. Results do not depend on it, except
                        the FISTA restart product's summation order.        */
} rihv_options;

/* One detected particle (Section 2, segmentation paragraph). */
typedef struct {
  double cx, cy, cz;  /* |x|-weighted centroid in voxel units (x, y, z)     */
  double weight;      /* sum of |x| over the component                       */
  int64_t first;      /* smallest linear voxel index (k*ny + j)*nx + i       */
  int32_t nvox;       /* voxels in the component                             */
  int32_t pad_;
} rihv_particle;

/* Fills *opt with the defaults listed above. */
void rihv_default_options(rihv_options* opt);

/* Creates a handle for one grid and optics (lengths in metres; wavelength is
 * the illumination wavelength, not a regularisation weight). Allocates all
 * scratch for forward/adjoint/prox/solve on the current CUDA device.
 * Returns RIHV_ERR_UNSUPPORTED_SIZE for sizes outside the supported set,
 * RIHV_ERR_INVALID_ARG for non-positive wavelength/pitch or a null *out,
 * RIHV_ERR_OOM if scratch does not fit. */
rihv_status rihv_create(int nx, int ny, int nz, double wavelength, double pitch,
                        double z0, double dz, rihv_handle* out);

/* Synchronises the handle's stream, frees its scratch and the handle. */
rihv_status rihv_destroy(rihv_handle h);

/* Sets the cudaStream_t (passed as void*) all later calls queue on. */
rihv_status rihv_set_stream(rihv_handle h, void* stream);

/* Sets solver options (copied). Invalid values return RIHV_ERR_INVALID_ARG. */
rihv_status rihv_set_options(rihv_handle h, const rihv_options* opt);

/* Forward model (Section 2, linearised model b_hat = H x):
 * out = sum_j F^-1 (H_j . F x_j).
 * x: device complex64 [nz][ny][nx]; out: device complex64 [ny][nx]. */
rihv_status rihv_forward(rihv_handle h, const void* x, void* out);

/* Adjoint of the forward model ("reverse propagation", Section 2):
 * out_j = F^-1 (conj(H_j) . F r) for every plane j.
 * r: device complex64 [ny][nx]; out: device complex64 [nz][ny][nx]. */
rihv_status rihv_adjoint(rihv_handle h, const void* r, void* out);

/* Fused-lasso proximal operator (Section 2, FL paragraph): the TV prox of v
 * with weight t_tv by `inner_iters` Beck-Teboulle dual gradient-projection
 * steps from p = 0, then soft thresholding with t_l1. t_l1 and t_tv are
 * already multiplied by the step size. Uses the handle's tv_dims.
 * v, x_out: device complex64 [nz][ny][nx]. */
rihv_status rihv_prox_fused_lasso(rihv_handle h, const void* v, float t_l1, float t_tv,
                                  int inner_iters, void* x_out);

/* Fused-lasso FISTA (Section 2, FISTA paragraph and shrinkage step) for
 * `iters` iterations with step 1/L, L = 2 max_f sum_j |H_j(f)|^2.
 * hologram: host or device float32 [ny][nx].
 * x0_or_null: host or device complex64 volume to start from, or NULL for 0.
 * x_out: host or device complex64 [nz][ny][nx], receives x_iters.
 * objective_trace_or_null: host or device double array with one slot per
 *   objective check (iters / check_every entries), or NULL.
 * If *iters_done is non-NULL it receives the iterations actually run (fewer
 * than iters only when the f_star stop test fired). The call returns after
 * the stream has finished the solve; a non-finite objective or norm returns
 * RIHV_ERR_NONFINITE. Host buffers are read by the CPU, one byte per page,
 * just before the device copies them (x_out once the iterations have run):
 * without it the first device-to-host copy into pinned pages the CPU had
 * not touched for seconds ran several times slower. */
rihv_status rihv_solve(rihv_handle h, const float* hologram, float lambda_l1, float lambda_tv,
                       int iters, const void* x0_or_null, void* x_out,
                       double* objective_trace_or_null, int* iters_done);

/* Particle detection on a volume (Section 2, segmentation paragraph):
 * voxels with |x| > rel_thresh * max|x|, 26-connected components, components
 * of <= min_vox voxels dropped, |x|-weighted centroids. Particles are written
 * to host array `out` (capacity max_out) in order of their smallest linear
 * voxel index; *n_out receives the number found (which may exceed max_out;
 * only max_out are written). x: device complex64 [nz][ny][nx], or NULL for
 * the result of the last rihv_solve on this handle (which the library keeps
 * on the device even when x_out was host memory). Synchronises
 * the stream. The first call allocates the labelling scratch, and a call that
 * finds more components than any before grows the per-component buffers. */
rihv_status rihv_detect(rihv_handle h, const void* x, float rel_thresh, int min_vox,
                        rihv_particle* out, int max_out, int* n_out);

/* The same detection on a volume's per-plane COO form (Section 2: volumes
 * are stored plane by plane as lists of their non-zero elements; see
 * rihv_coo_compact for the layout), with work in proportion to the nnz
 * listed entries instead of the nx*ny*nz voxels: the threshold is taken over
 * the listed values (the maximum of |x| is the same), the entries above it
 * are compacted into an ascending list of linear voxel indices, and the
 * components are formed over that list, each entry finding its 26-neighbours
 * by binary search. Gives the particles rihv_detect gives on the expanded
 * volume (same components, order and sizes; centroids up to FP64 summation
 * order). plane_offsets: device int64 [nz+1], checked on the host first (0
 * first, nnz last, non-decreasing, at most nx*ny per plane; else
 * RIHV_ERR_INVALID_ARG). rows, cols: device int32 [nnz]; vals: device
 * complex64 [nnz] (16-byte aligned); nnz < 2^31 (else
 * RIHV_ERR_UNSUPPORTED_SIZE). nnz = 0 finds nothing. out, max_out, n_out as
 * for rihv_detect. Synchronises the stream; the first call (and one with
 * more entries than any before) allocates the list scratch. */
rihv_status rihv_detect_coo(rihv_handle h, const long long* plane_offsets, const int* rows,
                            const int* cols, const void* vals, long long nnz, float rel_thresh,
                            int min_vox, rihv_particle* out, int max_out, int* n_out);

/* Batched solves. A batch groups handles (each with its own grid, optics,
 * options and scratch; a handle may appear once) whose holograms are solved
 * together: rihv_batch_solve runs every handle's complete FISTA solve (the
 * same iteration count and lambdas for all) as one CUDA graph, one branch per
 * handle, so the kernels of different holograms run concurrently and no
 * launch returns to the host between iterations. The graph is captured on the
 * first call and reused while iters, the lambdas, the presence of x0s and the
 * handles' options and tuning stay the same. Not in the paper; it serves
 * time-resolved sequences (many holograms per measurement).
 * holograms[i]: host or device float32 hologram of handle i; x0s: NULL or an
 * array of host or device warm-start volumes; x_outs[i]: host or device
 * complex64 output volume; traces: NULL or per-handle host or device arrays
 * of iters / check_every doubles (NULL entries allowed). Handles whose
 * options set a stop test stop early inside the graph (see
 * rihv_batch_iterations); the others run `iters`. Each handle's volume and
 * trace are bitwise equal to those of its own rihv_solve (inside the graph the
 * TV launches before the last one of each prox run on larger z-chunks, which
 * changes no result). The call returns after the batch has finished. */
typedef struct rihv_batch_st* rihv_batch;
rihv_status rihv_batch_create(const rihv_handle* handles, int n, rihv_batch* out);
rihv_status rihv_batch_solve(rihv_batch b, const float* const* holograms, float lambda_l1,
                             float lambda_tv, int iters, const void* const* x0s_or_null,
                             void* const* x_outs, double* const* traces_or_null);
rihv_status rihv_batch_destroy(rihv_batch b);
/* Iterations each hologram of the batch ran in the last rihv_batch_solve
 * (iters_done: host int[n], in handle order). A handle whose options set a
 * stop test (f_star > 0, check_every > 0) stops at the first objective check
 * that meets F(x_k) <= f_star (1 + tol), exactly where rihv_solve stops: the
 * batch graph then runs its iterations in chunks of check_every, every chunk
 * after the first behind a conditional (IF) graph node whose condition the
 * previous chunk sets on the device; objective checks it does not reach read
 * as NaN in its trace. Without a stop test all holograms run `iters`. */
rihv_status rihv_batch_iterations(rihv_batch b, int* iters_done);

/* Autotuner (not in the paper). Times, on the handle's own scratch, the TV
 * kernel's z-chunk length (8..256 planes per CTA) and steps per launch (1 or
 * 2, i.e. halo depth), the number of planes each column-pass CTA sums
 * (z-group size), and the row-pass FFT tile (1, 2, 4 or 8 rows per CTA, for
 * power-of-two nx), then applies the fastest to the handle. With a non-NULL
 * cache_path the result is looked up first (key: nx ny nz tv_dims) and
 * appended after a search, one line per shape. chosen_or_null (int[4])
 * receives {z-chunk, steps per launch, planes per column group, rows per
 * row-pass CTA}. Synchronises; the scratch contents (x, y, v) are
 * overwritten. An option tv_zchunk > 0 overrides the tuned z-chunk. */
rihv_status rihv_autotune(rihv_handle h, const char* cache_path, int* chosen_or_null);

/* The z-chunking a two-step TV launch of a solve on this handle uses (not in
 * the paper): final = 0 for the launches that read the dual (and the first
 * of a prox), 1 for the fused-finalize launch. out3 receives {planes per
 * z-chunk, split_tile, planes per z-chunk from split_tile on (0: no split)}
 * (option tv_split). Host-only; no device work. */
rihv_status rihv_tv_schedule(rihv_handle h, int final, int* out3);

/* The split rule itself, without a handle or a device (not in the paper):
 * for an nx x ny x nz volume, a two-step TV launch (final = 1: the
 * fused-finalize tile) with z-chunks of `zchunk` planes on `sms` SMs, one
 * CTA per SM. out2 receives {split_tile, planes per z-chunk from split_tile
 * on}, {0, 0} when equal z-chunks are kept. Host computation only. */
rihv_status rihv_tv_split_plan(int nx, int ny, int nz, int final, int zchunk, int sms, int* out2);

/* Steps of the last rihv_solve run with the FASTA-style solver (option
 * solver = 1; not in the paper beyond its naming FASTA): the accepted step
 * size of every iteration, in order, into taus (host, first `capacity`
 * written), their number into *n_steps, and the number of backtracking
 * halvings into *backtracks (may be NULL). After a FISTA solve *n_steps is
 * that of the last FASTA solve on the handle (0 if none). */
rihv_status rihv_fasta_steps(rihv_handle h, double* taus, int capacity, int* n_steps,
                             int* backtracks);

/* Per-plane COO form of a volume (Section 2, GPU implementation paragraph:
 * volumes stored in the coordinate sparse format, every plane indexing its
 * own non-zero elements). An element is non-zero unless both its real and
 * imaginary parts are zero. Plane k's entries occupy [plane_offsets[k],
 * plane_offsets[k+1]) in row-major order (row j, then column i). rows and cols
 * are int32 and vals complex64: 16 bytes per entry (the paper counts 8-byte
 * indices, 24 bytes; int32 covers every supported plane size).
 *
 * rihv_coo_compact: x is device complex64 [nz][ny][nx] of the handle's shape,
 * or NULL for the last solve's result. plane_offsets: device int64 [nz+1],
 * always written. rows, cols, vals: device arrays of `capacity` entries (16-
 * byte aligned); *nnz (host) receives the number of non-zeros in every case.
 * With capacity < *nnz (e.g. 0 and NULL arrays, to query the size) no entry
 * is written and RIHV_ERR_INVALID_ARG is returned. Deterministic; synchronous
 * (it reads the count back). */
rihv_status rihv_coo_compact(rihv_handle h, const void* x_or_null, long long* plane_offsets,
                             int* rows, int* cols, void* vals, long long capacity,
                             long long* nnz);

/* Dense x_out (device complex64 [nz][ny][nx]) from a per-plane COO form with
 * nnz entries: zero everywhere except the listed elements. plane_offsets
 * (device int64 [nz+1]) are checked on the host before any work (0 first, nnz
 * last, non-decreasing, at most nx*ny per plane; else RIHV_ERR_INVALID_ARG). An
 * entry outside its plane is skipped and reported as RIHV_ERR_INVALID_ARG when
 * the call returns. Synchronous. */
rihv_status rihv_coo_expand(rihv_handle h, const long long* plane_offsets, const int* rows,
                            const int* cols, const void* vals, long long nnz, void* x_out);

/* Fused-lasso prox without any allocation. The paper has no counterpart to
 * this entry point; it exists for callers that cannot call cudaMalloc: hosts
 * that hand out device memory only from their own fixed arena (memory the
 * library took behind their back would be missing from it), and services
 * that stop allocating after start-up so that no request can fail, or wait
 * on a device-wide synchronisation, for lack of memory.
 *
 * It computes what rihv_prox_fused_lasso computes, up to FP32 rounding order
 * (tv_dims TV prox by inner_iters dual gradient-projection steps from p = 0,
 * then soft threshold with t_l1), without a handle. Its scratch (the dual variable) is a static
 * device array inside the library of 6 x 8 MiB + 256 B, reserved on every GPU
 * that loads the library until the process exits. Limits: nx even and >= 2,
 * ny, nz >= 1, nx*ny*nz <= 1,048,576 voxels; larger volumes return
 * RIHV_ERR_UNSUPPORTED_SIZE before any work is queued (rihv_last_error(NULL)
 * says why).
 *
 * v, x_out: distinct device complex64 [nz][ny][nx], 16-byte aligned, on the
 * current device (else RIHV_ERR_INVALID_ARG). stream: a cudaStream_t of the
 * current device, or NULL. The work is queued on
 * the stream and the call returns; it calls no cudaMalloc, cudaFree or other
 * allocating routine. The first call on each device looks up the scratch's
 * device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture. All calls share the one scratch array,
 * which keeps the last call's contents: calls that may overlap on the GPU
 * (different streams, or different host threads) race and must be serialised
 * by the caller. A bounded wait inside the TV kernels that gave up (see
 * rihv_selftest_bounded_wait) cannot be reported by the return code, because
 * the call returns before the kernels run: it fills x_out with NaN instead,
 * so a caller that needs to know checks x_out for NaN. */
rihv_status rihv_prox_fused_lasso_noalloc(const void* v, void* x_out, int nx, int ny, int nz,
                                          int tv_dims, float t_l1, float t_tv, int inner_iters,
                                          void* stream);

/* Self-test of failure detection (no counterpart in the paper). Every wait
 * of the library's kernels on an mbarrier (TMA tile arrival) is bounded: after
 * a fixed number of polls the kernel records the failure in a device flag,
 * lets its own copies in flight land (again bounded) and returns, and the
 * calling entry point reports RIHV_ERR_TIMEOUT. This call runs that bounded
 * wait on a barrier that nothing ever arrives on, with `polls` polls
 * (1..2^22), on the handle's stream, and synchronises it. Expected result:
 * RIHV_ERR_TIMEOUT, with the CUDA context still usable. RIHV_ERR_CUDA if the
 * barrier completed or a CUDA call failed; RIHV_ERR_INVALID_ARG for polls out
 * of range. */
rihv_status rihv_selftest_bounded_wait(rihv_handle h, int polls);

/* Per-stage timing. Kernel launches are always counted per stage. With
 * profiling level 1 (rihv_set_profiling(h, 1)) the library also records CUDA
 * events around its stages on the handle's stream; level 2 adds events around
 * every TV launch (stages 7-9), which costs a little time: an event between
 * two launches keeps the second from starting while the first drains. rihv_stage_times returns accumulated milliseconds (0
 * without profiling) and launch counts per stage, after synchronising the
 * stream, and resets both. Stages, in order: 0 forward, 1 adjoint + gradient
 * step, 2 TV dual steps, 3 finalize (soft threshold, momentum, restart),
 * 4 objective, 5 detection, 6 solve set-up (hologram spectrum, x_0, scalars);
 * then the TV launches of stage 2 by kind (one scope per launch, counted in
 * stage 2 too): 7 the first launch of a prox (p = 0), 8 launches reading p,
 * 9 the last launch with the fused finalize (its finalize is not in stage 3).
 * n is the capacity of both arrays (up to 10 are written); either may be
 * NULL. */
rihv_status rihv_set_profiling(rihv_handle h, int on);
rihv_status rihv_stage_times(rihv_handle h, double* ms, long long* launches, int n);

/* Step size tau = 1/L used by rihv_solve (host-computed in FP64). */
rihv_status rihv_step_size(rihv_handle h, double* tau);

/* Message for the last failing call on h (or a global message if h is NULL). */
const char* rihv_last_error(rihv_handle h);

#ifdef __cplusplus
}
#endif

#endif /* RIHV_H */
