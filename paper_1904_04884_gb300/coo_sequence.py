"""A time-resolved sequence whose reconstructed volumes are stored in their
per-plane COO form between frames (Section 2: volumes kept plane by plane as
lists of their non-zero elements, which is what lets the paper hold sequences
of 10^9-voxel reconstructions).

One handle holds the dense working state of one frame. Every frame's
solution is compacted to its COO form on the device (rihv_coo_compact) and
only that form is kept; the next frame starts FISTA from the previous
frame's solution expanded back from its COO form (rihv_coo_expand), the
natural warm start for time-resolved holograms whose particles move little
between frames. Particles are the workload's discs advected by a Lamb-Oseen
vortex about the volume's axis; holograms come from this library's forward
operator plus noise.

    python -m paper_1904_04884_gb300.coo_sequence --workload fista_giga_1024x1024x1024 \
        --frames 3 --iters 30
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import synth, workloads
from .rihv import Rihv


def frame_hologram(h, w, parts, noise_seed, dev):
    """b = 1 - |1 - H a|^2 + sigma n for the discs `parts` (float32 [ny][nx])."""
    vol = np.zeros(w.shape, np.float32)
    synth.rasterise_discs(vol, parts)
    a = torch.from_numpy(vol).to(dev).to(torch.complex64)
    del vol
    field = torch.empty((w.ny, w.nx), dtype=torch.complex64, device=dev)
    h.forward(a, field)
    del a
    noise = synth.Stream(noise_seed).normal(w.nx * w.ny)
    return synth.intensity_hologram(field.cpu().numpy().astype(np.complex128), w.sigma, noise)


def run(w=workloads.GIGA, frames=3, iters=None, warm=True, gamma=4000.0, log=print,
        keep=False):
    """Solves `frames` frames; returns per-frame and total figures (and, with
    keep, the stored COO forms and the last dense solution)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    iters = iters or w.iters
    h = Rihv(*w.optics_tuple())
    h.set_options(tv_dims=w.tv_dims, n_inner=w.n_inner, check_every=10)
    parts = w.discs()
    x = torch.empty(w.shape, dtype=torch.complex64, device=dev)
    x0 = torch.empty_like(x) if warm else None
    stored, rows = [], []
    for f in range(frames):
        b = frame_hologram(h, w, parts, 7000 + f, dev)
        start = None
        t0 = time.perf_counter()
        if warm and stored:
            h.coo_expand(*stored[-1], x0)
            start = x0
        trace = np.zeros(max(1, iters // 10))
        h.solve(b, w.lam_l1, w.lam_tv, iters, x, x0=start, trace=trace)
        t1 = time.perf_counter()
        coo = h.coo_compact(x)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        stored.append(coo)
        nnz = int(coo[1].numel())
        rows.append({"frame": f, "warm": start is not None, "solve_s": t1 - t0,
                     "compact_s": t2 - t1, "nnz": nnz, "coo_bytes": 16 * nnz + 8 * (w.nz + 1),
                     "objective": float(trace[-1]) if iters >= 10 else None})
        parts.x, parts.y = synth.lamb_oseen_advect(parts.x, parts.y, gamma, 0.15 * w.nx,
                                                   0.5 * w.nx, 0.5 * w.ny)
    dense = 8 * w.nvox
    res = {"workload": w.name, "frames": frames, "iters": iters, "warm_from_previous": warm,
           "dense_bytes_per_frame": dense,
           "stored_coo_bytes": sum(r["coo_bytes"] for r in rows),
           "stored_dense_bytes": dense * frames,
           "voxel_iter_s": w.nvox * iters * frames / sum(r["solve_s"] for r in rows),
           "per_frame": rows}
    log(json.dumps(res))
    if keep:
        res["_stored"] = stored
        res["_last"] = x
        res["_handle"] = h
    else:
        h.close()
    return res


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--workload", default=workloads.GIGA.name)
    p.add_argument("--frames", type=int, default=3)
    p.add_argument("--iters", type=int, default=None)
    p.add_argument("--cold", action="store_true", help="start every frame from zero")
    a = p.parse_args()
    run(workloads.ALL[a.workload], a.frames, a.iters, warm=not a.cold)


if __name__ == "__main__":
    main()
