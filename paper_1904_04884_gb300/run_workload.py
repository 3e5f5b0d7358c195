"""End-to-end run of one named workload: the seeded particle volume, its
hologram from this library's forward operator (b = 1 - |1 - H a|^2 + noise),
the fused-lasso FISTA solve with the workload's weights and iteration count,
and detection; prints one JSON line with the time, the throughput and how the
detections match the placed discs: a detection matches a disc when its
centroid lies within ``--match-xy`` pixels laterally and ``--match-z`` planes
axially of the disc's centre (holographic depth resolution is several planes,
so the axial window is the wider one).

    python -m paper_1904_04884_gb300.run_workload --workload paper_turbulence_512x512x700
    python -m paper_1904_04884_gb300.run_workload --workload fista_large_1024x1024x256
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import synth, workloads
from .rihv import Rihv


def match(parts, discs, tol_xy, tol_z):
    """(recall, precision): the fraction of discs with a detection inside the
    window, and of detections (fibres excluded from the truth) with a disc
    inside it."""
    from scipy.spatial import cKDTree
    if not len(parts) or not len(discs):
        return 0.0, 0.0
    c = np.array([p["centroid"] for p in parts], np.float64)        # x, y, z (voxel units)
    # disc centres are continuous (pixel i spans [i, i+1)); centroids are in
    # voxel indices, so move the centres by half a pixel
    t = np.stack([discs.x - 0.5, discs.y - 0.5, discs.z.astype(np.float64)], axis=1)
    scale = np.array([1.0 / tol_xy, 1.0 / tol_xy, 1.0 / tol_z])
    d_det, _ = cKDTree(t * scale).query(c * scale, p=np.inf)
    d_true, _ = cKDTree(c * scale).query(t * scale, p=np.inf)
    return float(np.mean(d_true <= 1.0)), float(np.mean(d_det <= 1.0))


def run(name, tv_dims=None, iters=None, lam_l1=None, lam_tv=None, tol_xy=2.0, tol_z=5.0,
        n_inner=None, skip_empty_planes=0):
    w = workloads.ALL[name]
    dev = torch.device("cuda:0")
    h = Rihv(*w.optics_tuple())
    n_inner = w.n_inner if n_inner is None else n_inner
    h.set_options(tv_dims=tv_dims or w.tv_dims, n_inner=n_inner, check_every=10,
                  skip_empty_planes=skip_empty_planes)
    t0 = time.perf_counter()
    a = torch.from_numpy(w.opacity().astype(np.complex64)).to(dev)
    field = torch.empty((w.ny, w.nx), dtype=torch.complex64, device=dev)
    h.rihv_forward(a, field)
    del a
    b = synth.intensity_hologram(field.cpu().numpy().astype(np.complex128), w.sigma,
                                 w.noise()).astype(np.float32)
    t_data = time.perf_counter() - t0
    b_dev = torch.from_numpy(b).to(dev)
    x = torch.empty(w.shape, dtype=torch.complex64, device=dev)
    n_it = iters or w.iters
    l1 = w.lam_l1 if lam_l1 is None else lam_l1
    ltv = w.lam_tv if lam_tv is None else lam_tv
    trace = np.zeros(n_it // 10)
    h.rihv_solve(b_dev, l1, ltv, 2, x)       # warm the kernels
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    n_run = h.rihv_solve(b_dev, l1, ltv, n_it, x, trace=trace)
    torch.cuda.synchronize()
    t_solve = time.perf_counter() - t0
    # the same solve again with stage events, for the split of its time
    h.stage_times()
    h.set_profiling(1)
    h.rihv_solve(b_dev, l1, ltv, n_it, x)
    torch.cuda.synchronize()
    stages = {k: round(v[0] / n_it, 4) for k, v in h.stage_times().items()
              if k in ("forward", "adjoint", "tv", "finalize", "objective") and v[1]}
    h.set_profiling(0)
    t0 = time.perf_counter()
    parts = h.rihv_detect(x, 2.0 / 256.0, 5)
    t_det = time.perf_counter() - t0
    recall, precision = match(parts, w.discs(), tol_xy, tol_z)
    off = h.rihv_coo_compact(x)[0].cpu().numpy()
    per_plane = np.diff(off)
    res = {"workload": w.name, "shape": list(w.shape), "iters": n_it,
           "tv_dims": tv_dims or w.tv_dims, "lam_l1": l1, "lam_tv": ltv, "n_inner": n_inner,
           "skip_empty_planes": skip_empty_planes, "stage_ms_per_iter": stages,
           "solve_s": t_solve, "voxel_iter_s": w.nvox * n_it / t_solve,
           "ms_per_iter": 1e3 * t_solve / n_it, "iters_run": n_run, "detect_s": t_det,
           "discs_placed": w.n_discs, "fibres_placed": w.n_fibres, "detected": len(parts),
           "match_window_px": [tol_xy, tol_xy, tol_z], "recall": recall, "precision": precision,
           "nonzeros": int(off[-1]), "planes_nonzero": int(np.count_nonzero(per_plane)),
           "objective_first_last": [float(trace[0]), float(trace[-1])] if len(trace) else None,
           "data_s": t_data}
    print(json.dumps(res), flush=True)
    return res


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--workload", default="paper_turbulence_512x512x700", choices=sorted(workloads.ALL))
    p.add_argument("--tv-dims", type=int, default=None, choices=[2, 3])
    p.add_argument("--iters", type=int, default=None)
    p.add_argument("--lam-l1", type=float, default=None)
    p.add_argument("--lam-tv", type=float, default=None)
    p.add_argument("--match-xy", type=float, default=2.0)
    p.add_argument("--match-z", type=float, default=5.0)
    p.add_argument("--n-inner", type=int, default=None)
    p.add_argument("--skip-empty-planes", type=int, default=0, choices=[0, 1])
    a = p.parse_args()
    run(a.workload, a.tv_dims, a.iters, a.lam_l1, a.lam_tv, a.match_xy, a.match_z, a.n_inner,
        a.skip_empty_planes)


if __name__ == "__main__":
    main()
