"""Benchmark of the fused-lasso FISTA reconstruction on one GB300 per rank.

One step = one complete reconstruction of the 1024 x 1024 x 256 particle-field
hologram (10,000 discs of 8 um and 200 fibres; 300 FISTA iterations, 20 TV
dual steps per prox, objective every 10 iterations, then particle
detection), all through the C ABI.

value  : voxel-iterations/s with hologram and volumes resident in HBM.
e2e    : the same metric with pinned HOST buffers: the hologram is copied in
         and the volume copied out inside rihv_solve, every step.
roofline: the TV dual-step kernel (the dominant kernel), from CUDA events the
         library records around every TV launch on its own stream during the
         last timed step; algorithmic bytes 56 per voxel for a launch reading p.
mid    : the same measurement on the 512 x 512 x 128 workload (200 iterations).
cpu_baseline: the FP64 oracle, as it stands, on the host cores: one process
         per core (spawned), each solving its own one-plane slab of the workload,
         and the same on one core.
time_to_tolerance: per-hologram time to F*(1+1e-3) on 20 held-out 256x256x64
         samples: plain FISTA, the learned warm start, batching, and both,
         every arm with its stop tests inside a CUDA graph.
batched: the time-resolved 64-frame sequence of mixed sizes (256^2 x 64,
         512^2 x 128, 768^2 x 192) as batched CUDA graphs against one frame
         at a time.
library_baseline: the same FISTA iteration on the same workload written
         with PyTorch operators (cuFFT plane transforms, stored transfer
         functions, one element-wise kernel per operation), the way the
         paper describes its own GPU code; two timed iterations.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank reconstructs its own hologram (independent work, no
data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

TV_PROFILE = os.path.join(ROOT, "profiles", "tv_step2_traffic_solve_512x512x128.json")
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--workload", default="fista_large_1024x1024x256",
                   help="named workload of the timed step (default: the 1024x1024x256 case)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--autotune", action="store_true",
                   help="run the library's autotuner on the handle before timing (at "
                        "1024x1024x256 it measured slower than the default tiles)")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the secondary measurements (mid workload, time to tolerance, "
                        "mixed-size sequence, library baseline)")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_hologram(b, w, rank):
    """Each rank reconstructs its own frame: rank 0 the workload's hologram,
    rank r > 0 the same with an added noise draw of its own (seed 1000 + r)."""
    if rank == 0:
        return b
    from paper_1904_04884_gb300 import synth
    return (b + w.sigma * synth.Stream(1000 + rank).normal(w.nx * w.ny).reshape(b.shape)
            ).astype(np.float32)


def max_over_ranks(pg, values):
    """Element-wise maximum of host float timings over all ranks (gloo)."""
    import torch
    t = torch.tensor(values, dtype=torch.float64)
    if pg:
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return [float(v) for v in t]


def job_value(vox_per_step, steps, world, ms):
    """Whole-job throughput: the units every rank processed over the slowest
    rank's time (weak scaling: each rank solves its own frame)."""
    return vox_per_step * steps * world / (ms / 1e3)


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # raw samples: RIHV_CLOCKS_DIR if set, else the system's temporary directory
        out_dir = os.environ.get("RIHV_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"rihv_clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1].split()[0]))
                mx = float(parts[2].split()[0])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        med = float(np.median(sm)) if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def _code_lines(path):
    """The lines of a C++ source with // comments and blank lines removed."""
    for line in open(path, encoding="utf-8"):
        code = line.split("//", 1)[0].rstrip()
        if code:
            yield code


def kernel_hash():
    """Hash of the TV kernel source and of the TV lines of the internal header
    (code only: comments do not count), so that the committed DRAM traffic is
    used only for the kernel it measured."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1904_04884_gb300", "csrc")
    for line in _code_lines(os.path.join(csrc, "tv_kernels.cu")):
        h.update(line.encode() + b"\n")
    for line in _code_lines(os.path.join(csrc, "rihv_internal.cuh")):
        if "Tv" in line or "TV" in line or "tv_" in line:
            h.update(line.encode() + b"\n")
    return h.hexdigest()[:16]


def measured_traffic(nvox, kernel):
    """DRAM bytes per launch of `kernel` (its launches reading p) from the
    committed ncu summary, scaled to this workload, or None when the kernel
    changed since it was captured."""
    try:
        prof = json.load(open(TV_PROFILE))
    except Exception:
        return None
    if prof.get("kernel_hash") != kernel_hash() or prof.get("kernel_name") != kernel:
        return None
    return prof["launch_kinds"]["tv_mid"]["dram_bytes_per_voxel"] * nvox




def hbm_peak():
    try:
        return float(json.load(open(PEAKS))["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def make_hologram(w, h, torch, dev):
    """Opacity volume from the seeded generator; hologram via this library's
    forward operator: b = 1 - |1 - H a|^2 + sigma n."""
    from paper_1904_04884_gb300 import synth
    a = torch.from_numpy(w.opacity().astype(np.complex64)).to(dev)
    field = torch.empty((w.ny, w.nx), dtype=torch.complex64, device=dev)
    h.forward(a, field)
    torch.cuda.synchronize()
    b = synth.intensity_hologram(field.cpu().numpy().astype(np.complex128), w.sigma, w.noise())
    del a
    return b


# ---------------------------------------------------------------------------
# The FP64 oracle on the host cores (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

def _oracle_slab(job):
    """One worker process: the oracle, as it stands, on its own slab of a
    workload (the slab's opacity, its hologram by the oracle's forward model,
    then `iters` FISTA iterations with the workload's weights and dual steps).
    Returns the wall-clock start and end of the FISTA iterations."""
    from oracle import rihv_oracle as O
    from paper_1904_04884_gb300 import synth, workloads
    wname, slab, iters = job
    w = workloads.ALL[wname]
    op = O.Optics(w.nx, w.ny, slab.shape[0], w.wavelength, w.pitch, w.z0, w.dz)
    b = synth.intensity_hologram(O.forward(slab.astype(np.float64), op), w.sigma, w.noise())
    t0 = time.time()
    O.fista(b.astype(np.float64), op, w.lam_l1, w.lam_tv, iters, w.n_inner, dims=w.tv_dims)
    return t0, time.time()


def host_cores():
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


class OraclePool:
    """`cores` spawned worker processes, one oracle slab each per round."""

    def __init__(self, w, cores, planes=1):
        import multiprocessing as mp
        self.w = w
        self.cores = cores
        vol = w.opacity()
        span = max(1, w.nz - planes + 1)
        self.slabs = [np.ascontiguousarray(vol[(i * planes) % span:(i * planes) % span + planes])
                      for i in range(cores)]
        self.vox = w.nx * w.ny * planes
        self.pool = mp.get_context("spawn").Pool(cores) if cores > 1 else None

    def run(self, iters, n=None):
        """One round on n slabs (all cores by default); returns the wall time
        from the first worker's start to the last one's end."""
        jobs = [(self.w.name, s, iters) for s in self.slabs[:n or self.cores]]
        res = self.pool.map(_oracle_slab, jobs, chunksize=1) if self.pool and len(jobs) > 1 \
            else [_oracle_slab(j) for j in jobs]
        return max(e for _, e in res) - min(s for s, _ in res)

    def close(self):
        if self.pool:
            self.pool.close()
            self.pool.join()


def cpu_baseline(w, iters=2):
    """The oracle on every host core (one spawned process per core, each
    solving its own one-plane slab of the workload for `iters` iterations)
    and on one core (one slab alone)."""
    cores = host_cores()
    pool = OraclePool(w, cores)
    try:
        pool.run(1, n=min(cores, 2))                  # workers up, modules imported
        t_all = pool.run(iters)
        t_one = pool.run(iters, n=1)
    finally:
        pool.close()
    value = cores * pool.vox * iters / t_all
    one = pool.vox * iters / t_one
    sample = (f"{iters} FISTA iterations (K={w.n_inner}) per process on its own "
              f"{w.nx}x{w.ny}x1 slab of the same workload, {cores} processes in parallel "
              f"({t_all:.1f} s wall); numpy FP64, one thread per process")
    return {"value": value, "unit": "voxel-iter/s", "cores": cores, "kind": "oracle",
            "sample": sample, "one_core": {"value": one, "cores": 1, "seconds": t_one}}


def run_reference(args, rank, world):
    """--impl reference: the FP64 oracle on the host cores, each step one
    FISTA iteration per core on its own one-plane slab of the same workload."""
    if rank != 0:
        return
    from paper_1904_04884_gb300 import workloads
    w = workloads.ALL[args.workload]
    cores = host_cores()
    pool = OraclePool(w, cores)
    try:
        for _ in range(args.warmup):
            pool.run(1)
        dt = sum(pool.run(1) for _ in range(args.steps))
    finally:
        pool.close()
    value = cores * pool.vox * args.steps / dt
    sample = (f"1 FISTA iteration (K={w.n_inner}) per process on its own {w.nx}x{w.ny}x1 slab "
              f"per step, {cores} processes")
    line = {
        "impl": "reference", "metric": "voxel-iterations/s", "value": value,
        "unit": "voxel-iter/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / max(1, args.steps), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "nx": w.nx, "ny": w.ny, "nz": w.nz, "iters": w.iters,
                   "tv_inner_steps": w.n_inner, "tv_dims": w.tv_dims,
                   "parallelism": f"replicas x{world}", "sample": sample},
        "cpu_baseline": {"value": value, "unit": "voxel-iter/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "voxel-iter/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Secondary measurements (one GPU)
# ---------------------------------------------------------------------------

def solve_rate(w, dev, steps=3, warmup=1):
    """Voxel-iterations/s of full solves (+ detection) of workload w, device
    buffers, CUDA events on the library's stream."""
    import torch
    from paper_1904_04884_gb300.rihv import Rihv
    stream = torch.cuda.Stream(device=dev)
    h = Rihv(*w.optics_tuple(), stream=stream)
    h.set_options(tv_dims=w.tv_dims, n_inner=w.n_inner, check_every=10)
    b = torch.from_numpy(make_hologram(w, h, torch, dev)).to(dev)
    x = torch.empty(w.shape, dtype=torch.complex64, device=dev)
    trace = torch.empty(max(1, w.iters // 10), dtype=torch.float64, device=dev)
    ndet = 0
    for _ in range(warmup):
        h.solve(b, w.lam_l1, w.lam_tv, w.iters, x, trace=trace)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        h.solve(b, w.lam_l1, w.lam_tv, w.iters, x, trace=trace)
        ndet = len(h.detect(x, 2.0 / 256.0, 5))
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    h.close()
    return {"workload": w.name, "value": w.nvox * w.iters * steps / (ms / 1e3),
            "unit": "voxel-iter/s", "ms_per_step": ms / steps, "steps": steps,
            "detections": ndet}


def time_to_tolerance(n_seeds=20, tol=1e-3, max_iters=400):
    """Per-hologram wall time to F* (1 + tol), checked every 10 iterations, on
    held-out 256x256x64 samples (seeds 20001...), F* the objective of a
    600-iteration plain solve. Four arms, every one with its stop tests inside
    a CUDA graph (conditional nodes, no host round trip): plain FISTA from
    zero one hologram at a time; the learned warm start one at a time
    (network inference included); plain FISTA with all holograms in one
    batched graph; warm start and batched graph together."""
    import torch
    from paper_1904_04884_gb300 import warmstart as W
    from paper_1904_04884_gb300.rihv import Batch
    from paper_1904_04884_gb300.unet import WarmStartUNet

    dev = torch.device("cuda:0")
    spec = W.SPEC
    net = WarmStartUNet.load(W.DEFAULT_WEIGHTS)
    h = W.handle(spec)
    seeds = list(range(20001, 20001 + n_seeds))
    samples = [W.make_sample(h, spec, s, dev) for s in seeds]
    f_star = [W.reference_objective(h, b, spec) for b, _ in samples]
    h.close()
    holos = [b for b, _ in samples]
    hs = [W.handle(spec, check_every=10, f_star=fs, tol=tol) for fs in f_star]
    x0s = [torch.empty(spec.shape, dtype=torch.complex64, device=dev) for _ in seeds]
    outs = [torch.empty(spec.shape, dtype=torch.complex64, device=dev) for _ in seeds]

    def predict_all():
        for (_, hb), x0 in zip(samples, x0s):
            net.predict(hb, x0)

    def timed(fn):
        fn()                                   # captures the graphs
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    t_inf = timed(predict_all) / n_seeds
    singles = [Batch([hh]) for hh in hs]

    def plain_single():
        for bt, b, x in zip(singles, holos, outs):
            bt.solve([b], spec.lam_l1, spec.lam_tv, max_iters, [x])

    def warm_single():
        for bt, b, x0, x in zip(singles, holos, x0s, outs):
            bt.solve([b], spec.lam_l1, spec.lam_tv, max_iters, [x], x0s=[x0])

    t_ps = timed(plain_single)
    it_plain = [bt.iterations()[0] for bt in singles]
    t_ws = timed(warm_single)
    it_warm = [bt.iterations()[0] for bt in singles]
    for bt in singles:
        bt.close()
    batch = Batch(hs)
    t_pb = timed(lambda: batch.solve(holos, spec.lam_l1, spec.lam_tv, max_iters, outs))
    it_pb = batch.iterations()
    t_wb = timed(lambda: batch.solve(holos, spec.lam_l1, spec.lam_tv, max_iters, outs, x0s=x0s))
    it_wb = batch.iterations()
    batch.close()
    for hh in hs:
        hh.close()
    assert net.errors() == 0
    plain, warm = t_ps / n_seeds, t_ws / n_seeds + t_inf
    pb, wb = t_pb / n_seeds, t_wb / n_seeds + t_inf
    return {"workload": "warmstart_256x256x64 (lambda 0.01 / 0.005, K = 20)",
            "tolerance": tol, "seeds": [seeds[0], seeds[-1]], "n_holograms": n_seeds,
            "plain_iters": it_plain, "warm_iters": it_warm,
            "plain_batched_iters": it_pb, "warm_batched_iters": it_wb,
            "mean_plain_iters": float(np.mean(it_plain)), "mean_warm_iters": float(np.mean(it_warm)),
            "inference_s_per_hologram": t_inf,
            "plain_s_per_hologram": plain, "warm_s_per_hologram": warm,
            "plain_batched_s_per_hologram": pb, "warm_batched_s_per_hologram": wb,
            "speedup_warm_only": plain / warm, "speedup_batch_only": plain / pb,
            "speedup": plain / wb}


class LibraryFista:
    """The fused-lasso FISTA iteration built the way the paper describes its
    own GPU code (Section 2, GPU implementation paragraph: a library FFT of
    every plane, the plane's transfer function applied in the spectrum,
    element-wise kernels for the rest), written with PyTorch operators:
    cuFFT for the 2D transforms, one element-wise kernel per operation, the
    transfer functions of all planes stored, the restart test read back to
    the host every iteration. Same method and FP32 complex arithmetic as the
    hand-written kernels, none of their fusion: a measured baseline for
    them. Nothing in the library uses it."""

    def __init__(self, w, device):
        import math

        import torch
        self.t = torch
        self.w = w
        f64 = torch.float64
        fx = torch.fft.fftfreq(w.nx, d=w.pitch, dtype=f64, device=device)
        fy = torch.fft.fftfreq(w.ny, d=w.pitch, dtype=f64, device=device)
        f2 = fy[:, None] ** 2 + fx[None, :] ** 2
        prop = (w.wavelength ** 2) * f2 < 1.0
        kappa = torch.sqrt(torch.where(prop, 1.0 / w.wavelength ** 2 - f2, torch.zeros_like(f2)))
        self.H = torch.empty(w.shape, dtype=torch.complex64, device=device)
        amp = prop.to(f64)
        for j in range(w.nz):          # plane by plane: FP64 phase modulo one cycle
            cyc = torch.remainder((w.z0 + j * w.dz) * kappa, 1.0)
            self.H[j] = torch.polar(amp, 2.0 * math.pi * cyc).to(torch.complex64)
        lip = 2.0 * float((self.H.abs() ** 2).sum(0).max())
        self.tau = 1.0 / lip if lip > 0 else 0.0

    def forward(self, x):
        fft = self.t.fft
        return fft.ifft2((self.H * fft.fft2(x)).sum(0))

    def adjoint(self, r):
        fft = self.t.fft
        return fft.ifft2(self.H.conj() * fft.fft2(r)[None])

    def _d(self, u, dims):
        t = self.t
        dx, dy, dz = t.zeros_like(u), t.zeros_like(u), t.zeros_like(u)
        dx[:, :, :-1] = u[:, :, 1:] - u[:, :, :-1]
        dy[:, :-1, :] = u[:, 1:, :] - u[:, :-1, :]
        if dims == 3:
            dz[:-1] = u[1:] - u[:-1]
        return dx, dy, dz

    def _dh(self, px, py, pz, dims):
        out = self.t.zeros_like(px)
        out[:, :, :-1] -= px[:, :, :-1]
        out[:, :, 1:] += px[:, :, :-1]
        out[:, :-1, :] -= py[:, :-1, :]
        out[:, 1:, :] += py[:, :-1, :]
        if dims == 3:
            out[:-1] -= pz[:-1]
            out[1:] += pz[:-1]
        return out

    def tv_prox(self, v, mu, k, dims):
        """K dual gradient-projection steps from p = 0, then v - mu D^H p."""
        t = self.t
        if mu == 0.0 or k == 0:
            return v.clone()
        p = [t.zeros_like(v) for _ in range(3)]
        step = 1.0 / (4.0 * dims * mu)
        for _ in range(k):
            g = self._d(v - mu * self._dh(*p, dims), dims)
            p = [pc + step * gc for pc, gc in zip(p, g)]
            norm = t.sqrt(sum(pc.real ** 2 + pc.imag ** 2 for pc in p))
            s = 1.0 / t.clamp(norm, min=1.0)
            p = [pc * s for pc in p]
        return v - mu * self._dh(*p, dims)

    def soft(self, u, kappa):
        t = self.t
        mag = u.abs()
        s = t.where(mag > kappa, 1.0 - kappa / t.clamp(mag, min=1e-30), t.zeros_like(mag))
        return u * s

    def solve(self, b, lam_l1, lam_tv, iters, k, dims, x0=None):
        """`iters` FISTA iterations (gradient restart on) from x0 or 0."""
        t = self.t
        tau = self.tau
        x_prev = t.zeros(self.w.shape, dtype=t.complex64, device=self.H.device) if x0 is None \
            else x0.clone()
        y, tk = x_prev.clone(), 1.0
        for _ in range(iters):
            v = y - (2.0 * tau) * self.adjoint(self.forward(y) - b)
            x = self.soft(self.tv_prox(v, tau * lam_tv, k, dims), tau * lam_l1)
            t_next = (1.0 + (1.0 + 4.0 * tk * tk) ** 0.5) / 2.0
            dx = x - x_prev
            if float((dx.conj() * (y - x)).real.sum()) > 0.0:
                t_next, y = 1.0, x.clone()
            else:
                y = x + ((tk - 1.0) / t_next) * dx
            x_prev, tk = x, t_next
        return x_prev


def library_baseline(w, b, dev, iters=2):
    """Voxel-iterations/s of `LibraryFista` on workload w (one untimed
    iteration first), CUDA events on the current stream."""
    import torch
    lf = LibraryFista(w, dev)
    bd = torch.from_numpy(np.asarray(b, np.float32)).to(dev).to(torch.complex64)
    lf.solve(bd, w.lam_l1, w.lam_tv, 1, w.n_inner, w.tv_dims)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    lf.solve(bd, w.lam_l1, w.lam_tv, iters, w.n_inner, w.tv_dims)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    return {"value": w.nvox * iters / (ms / 1e3), "unit": "voxel-iter/s",
            "ms_per_iteration": ms / iters, "iterations_timed": iters,
            "what": "the same FISTA iteration with PyTorch operators: cuFFT plane transforms, "
                    "stored transfer functions, one element-wise kernel per operation"}


def mixed_sequence(frames=64, iters=50, slots=4):
    """The time-resolved mixed-size sequence: batched graphs against one frame
    at a time (paper_1904_04884_gb300.sequence)."""
    from paper_1904_04884_gb300 import sequence
    r = sequence.run(frames, iters, slots, log=lambda *_: None)
    r.pop("hologram_seconds", None)
    return r


def main():
    args = parse()
    rank, world, local = dist_env()
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        pg = dist
    if args.impl == "reference":
        run_reference(args, rank, world)
        if pg:
            pg.barrier()
        return

    import torch
    from paper_1904_04884_gb300 import workloads
    from paper_1904_04884_gb300.rihv import Rihv

    assert torch.cuda.is_available(), "bench.py needs a GPU"
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workloads.ALL[args.workload]
    stream = torch.cuda.Stream(device=dev)
    h = Rihv(*w.optics_tuple(), stream=stream)
    h.set_options(tv_dims=w.tv_dims, n_inner=w.n_inner, check_every=10)
    tuned = None
    if args.autotune:
        # the library's autotuner on this handle (before any timing): TV z-chunk and
        # steps per launch, column-pass z-groups, row-pass FFT tile
        zc, per_l, zpg, rows = h.autotune()
        tuned = {"tv_zchunk": zc, "tv_steps_per_launch": per_l, "col_planes_per_group": zpg,
                 "fft_rows_per_cta": rows}

    b = rank_hologram(make_hologram(w, h, torch, dev), w, rank)
    b_dev = torch.from_numpy(b).to(dev)
    x_dev = torch.empty(w.shape, dtype=torch.complex64, device=dev)
    trace = torch.empty(w.iters // 10, dtype=torch.float64, device=dev)

    def step_device():
        h.solve(b_dev, w.lam_l1, w.lam_tv, w.iters, x_dev, trace=trace)
        return h.detect(x_dev, 2.0 / 256.0, 5)

    for _ in range(args.warmup):
        step_device()
    torch.cuda.synchronize()
    h.stage_times()                      # reset counters
    h.set_profiling(True)

    sampler = ClockSampler(local)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    sampler.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    ndet = 0
    for i in range(args.steps):
        # per-launch TV events (level 2) only in the last timed step: they put
        # a small gap between launches, so the other steps run without them
        if i == args.steps - 1:
            h.set_profiling(2)
        ndet = len(step_device())
    ev1.record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    stages = h.stage_times()
    h.set_profiling(False)

    # End to end through the public call with pinned host buffers.
    b_host = torch.from_numpy(b).pin_memory()
    x_host = torch.empty(w.shape, dtype=torch.complex64).pin_memory()
    trace_host = np.zeros(w.iters // 10)

    def step_host():
        h.solve(b_host, w.lam_l1, w.lam_tv, w.iters, x_host, trace=trace_host)
        return h.detect(None, 2.0 / 256.0, 5)     # detection on the solve's own result

    step_host()
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    t0 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 3))
    for _ in range(e2e_steps):
        step_host()
    e2e_s = time.perf_counter() - t0

    ms, e2e_ms = max_over_ranks(pg, [ms, e2e_s * 1e3])

    if rank != 0:
        return
    vox_iters = w.nvox * w.iters
    value = job_value(vox_iters, args.steps, world, ms)
    e2e_value = job_value(vox_iters, e2e_steps, world, e2e_ms)

    # Roofline of the dominant kernel, the TV launch that reads p (two dual
    # steps per launch by default), from the per-launch CUDA events the
    # library records on its stream during the last timed step. Algorithmic bytes
    # per voxel by launch kind: 56 reading p (read v and p, write p), 32 for
    # the first launch of a prox (p = 0: read v, write p), 64 for the last
    # launch with the fused finalize (read v, p, x_{k-1}, y_k; write x_k and
    # y_{k+1} instead of p).
    per = tuned["tv_steps_per_launch"] if tuned else h.options.tv_steps_per_launch
    tv_kernel = "k_tv_step2" if per == 2 else "k_tv_step"
    peak, peak_kind = hbm_peak()
    kinds = {}
    for kind, alg in (("tv_first", 32), ("tv_mid", 56), ("tv_final", 64)):
        kms, kn = stages[kind]
        kn = kn / args.steps         # launches are counted in every step, timed in the last
        if kn:
            avg_s = kms / 1e3 / kn
            ach = w.nvox * alg / avg_s / 1e9
            kinds[kind] = {"launches_timed": kn, "avg_launch_ms": avg_s * 1e3,
                           "alg_bytes_per_voxel": alg, "achieved_gbs": ach, "frac": ach / peak}
    dom = kinds.get("tv_mid") or kinds.get("tv_first")
    achieved = dom["achieved_gbs"] if dom else None
    alg_bytes_per_launch = w.nvox * (dom["alg_bytes_per_voxel"] if dom else 0)
    avg_launch_s = dom["avg_launch_ms"] / 1e3 if dom else 0.0
    main_stages = ("forward", "adjoint", "tv", "finalize", "objective", "detect", "setup")
    total_launches = sum(stages[k][1] for k in main_stages)

    # per-plane COO form of the solution (Section 2 sparse storage): size and
    # the time of a compaction and an expansion (synchronous calls)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    off, rows, cols, vals = h.coo_compact(x_dev)
    t1 = time.perf_counter()
    back = torch.empty_like(x_dev)
    h.coo_expand(off, rows, cols, vals, back)
    t2 = time.perf_counter()
    nnz = int(rows.numel())
    coo = {"nnz": nnz, "sparsity": 1.0 - nnz / w.nvox, "bytes": 16 * nnz + 8 * (w.nz + 1),
           "dense_bytes": 8 * w.nvox, "compact_ms": (t1 - t0) * 1e3, "expand_ms": (t2 - t1) * 1e3,
           "round_trip_exact": bool(torch.equal(back, x_dev))}
    del back, rows, cols, vals, b_host, x_host
    h.close()
    del x_dev, b_dev
    torch.cuda.empty_cache()

    mid = ttt = batched = library = None
    if not args.no_extras and world == 1:
        if w.name != workloads.MID.name:
            mid = solve_rate(workloads.MID, dev)
        torch.cuda.empty_cache()
        ttt = time_to_tolerance()
        torch.cuda.empty_cache()
        batched = mixed_sequence()
        torch.cuda.empty_cache()
        try:
            library = library_baseline(w, b, dev)
        except Exception as e:       # a failed baseline must not cost the bench line
            library = {"error": f"{type(e).__name__}: {e}"[:300]}
        torch.cuda.empty_cache()

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(w)

    line = {
        "metric": "voxel-iterations/s", "value": value, "unit": "voxel-iter/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64 (f32 complex, f64 reductions)", "data": "synthetic",
        "config": {"workload": w.name, "nx": w.nx, "ny": w.ny, "nz": w.nz, "iters": w.iters,
                   "tv_inner_steps": w.n_inner, "tv_dims": w.tv_dims,
                   "step": "full FISTA solve + objective every 10 iters + detection",
                   "l2": f"inputs larger than L2 ({8 * w.nvox / 1e6:.0f} MB per volume)",
                   "detections": ndet, "parallelism": f"replicas x{world}",
                   "tuned": tuned},
        "e2e": {"value": e2e_value, "unit": "voxel-iter/s", "steps": e2e_steps,
                "h2d_bytes_per_step": int(w.nx * w.ny * 4),
                "d2h_bytes_per_step": int(w.nvox * 8 + (w.iters // 10) * 8)},
        "gpu_launches": int(total_launches),
        "roofline": {"bound": "hbm", "kernel": tv_kernel + " (launch reading p)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None,
                     "traffic": measured_traffic(w.nvox, tv_kernel), "peak_kind": peak_kind,
                     "alg_bytes_per_launch": alg_bytes_per_launch,
                     "dual_steps_per_launch": per,
                     "avg_launch_ms": avg_launch_s * 1e3,
                     "tv_launch_kinds": kinds},
        "stages_ms_per_step": {k: stages[k][0] / args.steps for k in main_stages},
        "mid": mid,
        "time_to_tolerance": ttt,
        "batched": batched,
        "library_baseline": library,
        "coo": coo,
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
