"""Time-resolved hologram sequences of mixed sizes solved through batched CUDA
graphs, against the same frames solved one at a time.

Frames cycle through three sizes (256x256x64, 512x512x128, 768x768x192 at 5 um
pitch, 532 nm, z0 5 mm, 50 um planes). Each size has its own particle field
(500-3,000 opaque discs of 8-20 um) advected from frame to frame by a
Lamb-Oseen vortex of random circulation about the volume's axis. Holograms
come from this library's forward operator plus noise. Frames are solved in
groups: one handle per (size, slot), all of a group's frames captured as one
batched CUDA graph, replayed for every group.

    python -m paper_1904_04884_gb300.sequence --frames 64 --iters 50 --slots 4
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import synth
from .rihv import Batch, Rihv

SIZES = ((256, 256, 64), (512, 512, 128), (768, 768, 192))
OPTICS = dict(wavelength=532e-9, pitch=5e-6, z0=5e-3, dz=50e-6)


def frames(n_frames, seed=0):
    """Seeded opacity volumes (float32 [nz][ny][nx]) of the sequence, frame f
    of size f % 3; yields (size index, volume, noise sigma, noise seed)."""
    st = synth.Stream(seed)
    fields = []
    for nx, ny, nz in SIZES:
        n = int(st.integers(1, 2501)[0]) + 500
        parts = synth.random_discs(st, (nz, ny, nx), n, 8.0, 20.0, OPTICS["pitch"] * 1e6, False)
        gamma = float(st.uniform(1, 2000.0, 8000.0)[0])       # px^2 per frame
        fields.append([parts, gamma])
    for f in range(n_frames):
        k = f % len(SIZES)
        nx, ny, nz = SIZES[k]
        parts, gamma = fields[k]
        vol = np.zeros((nz, ny, nx), np.float32)
        synth.rasterise_discs(vol, parts)
        yield k, vol, 0.02, 5000 + f
        parts.x, parts.y = synth.lamb_oseen_advect(parts.x, parts.y, gamma, 0.15 * nx,
                                                   0.5 * nx, 0.5 * ny)


def hologram(h, vol, sigma, noise_seed, dev):
    a = torch.from_numpy(vol.astype(np.complex64)).to(dev)
    field = torch.empty(vol.shape[1:], dtype=torch.complex64, device=dev)
    h.forward(a, field)
    noise = synth.Stream(noise_seed).normal(field.numel())
    return synth.intensity_hologram(field.cpu().numpy().astype(np.complex128), sigma,
                                    noise).astype(np.float32)


def run(n_frames=64, iters=50, slots=4, lam_l1=0.01, lam_tv=0.005, n_inner=20, log=print):
    dev = torch.device("cuda:0")
    handles = [[Rihv(nx, ny, nz, **OPTICS) for _ in range(slots)] for nx, ny, nz in SIZES]
    for row in handles:
        for h in row:
            h.set_options(n_inner=n_inner, check_every=0)
    t0 = time.perf_counter()
    seq = [(k, hologram(handles[k][0], vol, s, ns, dev)) for k, vol, s, ns in frames(n_frames)]
    t_gen = time.perf_counter() - t0
    outs = [[torch.empty((nz, ny, nx), dtype=torch.complex64, device=dev) for _ in range(slots)]
            for nx, ny, nz in SIZES]
    vox = sum(SIZES[k][0] * SIZES[k][1] * SIZES[k][2] for k, _ in seq) * iters

    # groups: up to `slots` frames of every size per batched graph
    groups, cur, used = [], [], [0] * len(SIZES)
    for k, b in seq:
        if used[k] == slots:
            groups.append(cur)
            cur, used = [], [0] * len(SIZES)
        cur.append((k, used[k], b))
        used[k] += 1
    if cur:
        groups.append(cur)
    batches = {}

    def solve_group(g):
        key = tuple((k, s) for k, s, _ in g)
        if key not in batches:
            batches[key] = Batch([handles[k][s] for k, s, _ in g])
        batches[key].solve([b for _, _, b in g], lam_l1, lam_tv, iters,
                           [outs[k][s] for k, s, _ in g])

    for g in groups:                      # capture every distinct group's graph
        solve_group(g)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for g in groups:
        solve_group(g)
    torch.cuda.synchronize()
    t_batched = time.perf_counter() - t0

    for k, b in seq[:3]:                   # warm the one-at-a-time path
        handles[k][0].solve(b, lam_l1, lam_tv, 2, outs[k][0])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k, b in seq:
        handles[k][0].solve(b, lam_l1, lam_tv, iters, outs[k][0])
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    for bt in batches.values():
        bt.close()
    res = {"frames": n_frames, "sizes": [list(s) for s in SIZES], "iters": iters, "slots": slots,
           "groups": len(groups), "hologram_seconds": t_gen,
           "batched_s": t_batched, "sequential_s": t_seq,
           "batched_voxel_iter_s": vox / t_batched, "sequential_voxel_iter_s": vox / t_seq,
           "batched_frames_per_s": n_frames / t_batched, "speedup": t_seq / t_batched}
    log(json.dumps(res))
    return res


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--frames", type=int, default=64)
    p.add_argument("--iters", type=int, default=50)
    p.add_argument("--slots", type=int, default=4)
    a = p.parse_args()
    run(a.frames, a.iters, a.slots)


if __name__ == "__main__":
    main()
