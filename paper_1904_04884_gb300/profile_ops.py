"""Runs one library operator repeatedly on a seeded random input, for
profilers (ncu) and quick timing.

python -m paper_1904_04884_gb300.profile_ops --op prox --nx 256 --ny 256 --nz 64 --reps 3
ops: forward, adjoint, prox (fused-lasso prox with --inner TV steps), solve,
unet (warm-start network inference), unet_train (one training step).
"""
from __future__ import annotations

import argparse
import time

import numpy as np


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--op", default="prox",
                   choices=["forward", "adjoint", "prox", "solve", "unet", "unet_train"])
    p.add_argument("--nx", type=int, default=256)
    p.add_argument("--ny", type=int, default=256)
    p.add_argument("--nz", type=int, default=64)
    p.add_argument("--inner", type=int, default=20)
    p.add_argument("--iters", type=int, default=10)
    p.add_argument("--reps", type=int, default=3)
    p.add_argument("--tv-per-launch", type=int, default=2, choices=[1, 2],
                   help="dual TV steps per kernel launch (library default 2)")
    a = p.parse_args()

    import torch
    from paper_1904_04884_gb300 import synth
    from paper_1904_04884_gb300.rihv import Rihv

    dev = torch.device("cuda:0")
    h = Rihv(a.nx, a.ny, a.nz, 532e-9, 5e-6, 5e-3, 50e-6)
    h.set_options(tv_steps_per_launch=a.tv_per_launch)
    shape = (a.nz, a.ny, a.nx)
    g = synth.Stream(1).normal(2 * a.nx * a.ny * a.nz).astype(np.float32).view(np.complex64)
    vol = torch.from_numpy(g.reshape(shape)).to(dev)
    out = torch.empty_like(vol)
    plane = torch.empty((a.ny, a.nx), dtype=torch.complex64, device=dev)
    holo = torch.from_numpy(np.ones((a.ny, a.nx), np.float32)).to(dev)

    net = None
    if a.op.startswith("unet"):
        from paper_1904_04884_gb300.unet import WarmStartUNet
        net = WarmStartUNet((a.nz, a.ny, a.nx), seed=0)

    def once():
        if a.op == "unet":
            net.predict(vol, out)
        elif a.op == "unet_train":
            net.train_step(vol, out)
        elif a.op == "forward":
            h.forward(vol, plane)
        elif a.op == "adjoint":
            h.adjoint(plane, out)
        elif a.op == "prox":
            h.prox_fused_lasso(vol, 0.01, 0.005, a.inner, out)
        else:
            h.set_options(n_inner=a.inner, check_every=0, tv_steps_per_launch=a.tv_per_launch)
            h.solve(holo, 0.01, 0.005, a.iters, out)

    once()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(a.reps):
        once()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / a.reps
    print(f"{a.op} {a.nx}x{a.ny}x{a.nz}: {dt * 1e3:.3f} ms per call")


if __name__ == "__main__":
    main()
