"""Training and evaluation of the learned FISTA warm start (WarmStartUNet).

Samples are seeded synthetic particle volumes of 256 x 256 x 64 voxels
(200-2,000 opaque discs of 8-20 um, hologram noise sigma 0.01-0.03) with the
optics of the 512x512 workload (5 um pitch, 532 nm, z0 5 mm, dz 50 um).
Holograms come from this library's forward operator, the network input is
the back-propagated hologram H^H b (rihv_adjoint), and the training target is
the fused-lasso FISTA solution x* of that hologram (rihv_solve) minus FISTA's
first iterate from zero (2 tau H^H b), so the network learns the correction
that FISTA would otherwise build over many iterations.

    python -m paper_1904_04884_gb300.warmstart train --n-train 256 --epochs 8 \
        --out paper_1904_04884_gb300/weights/warmstart_256x256x64.npz
    python -m paper_1904_04884_gb300.warmstart eval --weights <file> --seeds 20001 20002
"""
from __future__ import annotations

import argparse
import json
import os
import time
from dataclasses import dataclass

import numpy as np
import torch

from . import synth
from .rihv import Rihv
from .unet import WarmStartUNet

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "weights", "warmstart_256x256x64.npz")


@dataclass(frozen=True)
class SampleSpec:
    nx: int = 256
    ny: int = 256
    nz: int = 64
    wavelength: float = 532e-9
    pitch: float = 5e-6
    z0: float = 5e-3
    dz: float = 50e-6
    lam_l1: float = 0.01
    lam_tv: float = 0.005
    n_inner: int = 20
    target_iters: int = 200

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)


SPEC = SampleSpec()


def discs(spec: SampleSpec, seed: int):
    """The seeded sample's discs (200-2,000 of 8-20 um) and hologram noise sigma."""
    st = synth.Stream(seed)
    n = int(st.integers(1, 1801)[0]) + 200
    sigma = float(st.uniform(1, 0.01, 0.03)[0])
    return synth.random_discs(st, spec.shape, n, 8.0, 20.0, spec.pitch * 1e6, False), sigma


def opacity(spec: SampleSpec, seed: int):
    """Seeded opacity volume of the sample's discs; returns (vol, sigma)."""
    parts, sigma = discs(spec, seed)
    vol = np.zeros(spec.shape, np.float32)
    synth.rasterise_discs(vol, parts)
    return vol, sigma


def make_sample(h: Rihv, spec: SampleSpec, seed: int, dev):
    """(hologram b float32 [ny][nx] on host, H^H b complex64 on device)."""
    vol, sigma = opacity(spec, seed)
    a = torch.from_numpy(vol.astype(np.complex64)).to(dev)
    field = torch.empty((spec.ny, spec.nx), dtype=torch.complex64, device=dev)
    h.forward(a, field)
    noise = synth.Stream(seed + 0x5EED).normal(spec.nx * spec.ny)
    b = synth.intensity_hologram(field.cpu().numpy().astype(np.complex128), sigma, noise)
    bc = torch.from_numpy(b.astype(np.complex64)).to(dev)
    hb = torch.empty(spec.shape, dtype=torch.complex64, device=dev)
    h.adjoint(bc, hb)
    return b, hb


def handle(spec: SampleSpec, check_every=0, **opts):
    h = Rihv(spec.nx, spec.ny, spec.nz, spec.wavelength, spec.pitch, spec.z0, spec.dz)
    h.set_options(n_inner=spec.n_inner, check_every=check_every, **opts)
    return h


def train(n_train=256, epochs=8, lr=1e-3, seed0=1, out=DEFAULT_WEIGHTS, spec=SPEC, log=print):
    dev = torch.device("cuda:0")
    h = handle(spec)
    t0 = time.time()
    data = []
    for s in range(seed0, seed0 + n_train):
        b, hb = make_sample(h, spec, s, dev)
        x = torch.empty(spec.shape, dtype=torch.complex64, device=dev)
        h.solve(b, spec.lam_l1, spec.lam_tv, spec.target_iters, x)
        data.append((hb, x))
    torch.cuda.synchronize()
    t_data = time.time() - t0
    net = WarmStartUNet((spec.nz, spec.ny, spec.nx), seed=seed0)
    net.base_coeff = float(2.0 * h.step_size())
    # targets: the correction to FISTA's first iterate (data preparation)
    data = [(hb, (x - net.base_coeff * hb).contiguous()) for hb, x in data]
    k = min(16, n_train)
    net.scale_in = float(1.0 / np.mean([hb.abs().pow(2).mean().sqrt().item() for hb, _ in data[:k]]))
    net.scale_out = float(np.mean([x.abs().pow(2).mean().sqrt().item() for _, x in data[:k]]))
    order = np.arange(n_train)
    rng = np.random.default_rng(seed0)
    losses = []
    t1 = time.time()
    for ep in range(epochs):
        rng.shuffle(order)
        ep_loss = 0.0
        for i in order:
            hb, x = data[i]
            lr_now = lr * (0.5 ** (ep // max(1, epochs // 3)))
            ep_loss += net.train_step(hb, x, lr_now).item()
        losses.append(ep_loss / n_train)
        log(f"epoch {ep}: mean loss {losses[-1]:.5f}")
    torch.cuda.synchronize()
    t_train = time.time() - t1
    assert net.errors() == 0, "a convolution kernel's bounded wait gave up"
    os.makedirs(os.path.dirname(out), exist_ok=True)
    net.save(out)
    info = {"n_train": n_train, "epochs": epochs, "lr": lr, "losses": losses,
            "lam_l1": spec.lam_l1, "lam_tv": spec.lam_tv, "target_iters": spec.target_iters,
            "data_seconds": t_data, "train_seconds": t_train,
            "steps": n_train * epochs, "ms_per_step": 1e3 * t_train / (n_train * epochs)}
    with open(os.path.splitext(out)[0] + ".json", "w") as f:
        json.dump(info, f, indent=1)
    return net, info


def iterations_to_tolerance(h, b, spec, x0=None, f_star=None, tol=1e-3, max_iters=600):
    """FISTA iterations (checked every 10) until F(x_k) <= F* (1 + tol), and the
    wall time of that solve."""
    dev = torch.device("cuda:0")
    x = torch.empty(spec.shape, dtype=torch.complex64, device=dev)
    h.set_options(n_inner=spec.n_inner, check_every=10, f_star=float(f_star), tol=tol)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    done = h.solve(b, spec.lam_l1, spec.lam_tv, max_iters, x, x0=x0)
    torch.cuda.synchronize()
    return done, time.perf_counter() - t0, x


def reference_objective(h, b, spec, iters=600):
    trace = np.zeros(iters // 10)
    x = torch.empty(spec.shape, dtype=torch.complex64, device="cuda:0")
    h.set_options(n_inner=spec.n_inner, check_every=10)
    h.solve(b, spec.lam_l1, spec.lam_tv, iters, x, trace=trace)
    return float(trace.min())


def evaluate(weights=DEFAULT_WEIGHTS, seeds=(20001, 20002, 20003), spec=SPEC, tol=1e-3):
    """Iterations and time to F*(1+tol) from zero and from the network's x0."""
    dev = torch.device("cuda:0")
    net = WarmStartUNet.load(weights)
    h = handle(spec)
    rows = []
    for s in seeds:
        b, hb = make_sample(h, spec, s, dev)
        f_star = reference_objective(h, b, spec)
        it0, t0, _ = iterations_to_tolerance(h, b, spec, None, f_star, tol)
        x0 = torch.empty(spec.shape, dtype=torch.complex64, device=dev)
        torch.cuda.synchronize()
        ti = time.perf_counter()
        net.predict(hb, x0)
        torch.cuda.synchronize()
        t_inf = time.perf_counter() - ti
        it1, t1, _ = iterations_to_tolerance(h, b, spec, x0, f_star, tol)
        rows.append({"seed": s, "f_star": f_star, "plain_iters": it0, "plain_s": t0,
                     "warm_iters": it1, "warm_s": t1 + t_inf, "inference_s": t_inf})
    return rows


def main():
    p = argparse.ArgumentParser()
    sub = p.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train")
    t.add_argument("--n-train", type=int, default=256)
    t.add_argument("--epochs", type=int, default=8)
    t.add_argument("--lr", type=float, default=1e-3)
    t.add_argument("--out", default=DEFAULT_WEIGHTS)
    e = sub.add_parser("eval")
    e.add_argument("--weights", default=DEFAULT_WEIGHTS)
    e.add_argument("--seeds", type=int, nargs="+", default=[20001, 20002, 20003])
    for q in (t, e):
        q.add_argument("--lam-l1", type=float, default=SPEC.lam_l1)
        q.add_argument("--lam-tv", type=float, default=SPEC.lam_tv)
    a = p.parse_args()
    spec = SampleSpec(lam_l1=a.lam_l1, lam_tv=a.lam_tv)
    if a.cmd == "train":
        _, info = train(a.n_train, a.epochs, a.lr, out=a.out, spec=spec)
        print(json.dumps(info))
    else:
        print(json.dumps(evaluate(a.weights, a.seeds, spec=spec)))


if __name__ == "__main__":
    main()
