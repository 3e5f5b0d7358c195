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


def train_stream(seeds=range(1, 10001), init=DEFAULT_WEIGHTS, out=DEFAULT_WEIGHTS, group=16,
                 lr0=3e-4, lr1=3e-5, eval_seeds=range(20001, 20021),
                 eval_every=2000, final_eval_seeds=range(20001, 20101), time_limit_s=None,
                 spec=SPEC, log=print):
    """Continues training from `init` over fresh samples, each used once: the
    samples of `seeds` are generated in groups of `group`, their FISTA targets
    solved together in one batched CUDA graph, then one Adam step per sample
    (learning rate decaying linearly from lr0 to lr1). Every `eval_every`
    samples (and before the first) the iterations to F* (1 + 1e-3) from the
    network's start are measured on `eval_seeds`; at the end on
    `final_eval_seeds`. Weights go to `out` (and `out` + '.ckpt.npz' at each
    evaluation); the record to the same name with .json."""
    from .rihv import Batch
    dev = torch.device("cuda:0")
    net = WarmStartUNet.load(init)
    hs = [handle(spec) for _ in range(group)]
    batch = Batch(hs)
    outs = [torch.empty(spec.shape, dtype=torch.complex64, device=dev) for _ in range(group)]
    h_eval = handle(spec)
    ref = {}

    def curve(eval_list):
        rows = []
        for s in eval_list:
            if s not in ref:
                b, hb = make_sample(h_eval, spec, s, dev)
                fs = reference_objective(h_eval, b, spec)
                it0, _, _ = iterations_to_tolerance(h_eval, b, spec, None, fs)
                ref[s] = (b, hb, fs, it0)
            b, hb, fs, it0 = ref[s]
            x0 = torch.empty(spec.shape, dtype=torch.complex64, device=dev)
            net.predict(hb, x0)
            it1, _, _ = iterations_to_tolerance(h_eval, b, spec, x0, fs)
            rows.append((s, it0, it1))
        return {"plain_iters": [r[1] for r in rows], "warm_iters": [r[2] for r in rows],
                "mean_plain": float(np.mean([r[1] for r in rows])),
                "mean_warm": float(np.mean([r[2] for r in rows]))}

    seeds = list(seeds)
    t_start = time.time()
    record = {"init": os.path.basename(init), "seeds": [seeds[0], seeds[-1]], "group": group,
              "lr": [lr0, lr1], "target_iters": spec.target_iters, "curve": [], "losses": []}
    record["curve"].append({"samples": 0, **curve(eval_seeds)})
    log(json.dumps(record["curve"][-1]))
    done, loss_acc, loss_n = 0, torch.zeros(1, dtype=torch.float64, device=dev), 0
    stopped = False
    for g0 in range(0, len(seeds), group):
        chunk = seeds[g0:g0 + group]
        samples = [make_sample(hs[0], spec, s, dev) for s in chunk]
        holos = [b for b, _ in samples] + [samples[-1][0]] * (group - len(chunk))
        batch.solve(holos, spec.lam_l1, spec.lam_tv, spec.target_iters, outs)
        for (b, hb), x in zip(samples, outs):
            lr = lr0 + (lr1 - lr0) * done / max(1, len(seeds) - 1)
            loss_acc += net.train_step(hb, (x - net.base_coeff * hb).contiguous(), lr)
            loss_n += 1
            done += 1
        if done % 500 < group:
            record["losses"].append({"samples": done, "mean_loss": float(loss_acc.item()) / loss_n})
            loss_acc.zero_()
            loss_n = 0
        if done % eval_every < group or done == len(seeds):
            record["curve"].append({"samples": done, **curve(eval_seeds)})
            log(json.dumps(record["curve"][-1]))
            net.save(out + ".ckpt.npz")
        if time_limit_s and time.time() - t_start > time_limit_s:
            stopped = True
            break
    assert net.errors() == 0, "a convolution kernel's bounded wait gave up"
    batch.close()
    record["samples_trained"] = done
    record["stopped_at_time_limit"] = stopped
    record["train_seconds"] = time.time() - t_start
    record["final"] = {"seeds": [min(final_eval_seeds), max(final_eval_seeds)],
                       **curve(list(final_eval_seeds))}
    log(json.dumps(record["final"]))
    net.save(out)
    with open(os.path.splitext(out)[0] + ".stream.json", "w") as f:
        json.dump(record, f, indent=1)
    return record


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
    st = sub.add_parser("stream", help="continue training over fresh samples, each used once")
    st.add_argument("--first-seed", type=int, default=1)
    st.add_argument("--n", type=int, default=10000)
    st.add_argument("--init", default=DEFAULT_WEIGHTS)
    st.add_argument("--out", required=True)
    st.add_argument("--time-limit", type=float, default=None)
    e = sub.add_parser("eval")
    e.add_argument("--weights", default=DEFAULT_WEIGHTS)
    e.add_argument("--seeds", type=int, nargs="+", default=[20001, 20002, 20003])
    for q in (t, e):
        q.add_argument("--lam-l1", type=float, default=SPEC.lam_l1)
        q.add_argument("--lam-tv", type=float, default=SPEC.lam_tv)
    a = p.parse_args()
    if a.cmd == "stream":
        train_stream(range(a.first_seed, a.first_seed + a.n), a.init, a.out,
                     time_limit_s=a.time_limit)
        return
    spec = SampleSpec(lam_l1=a.lam_l1, lam_tv=a.lam_tv)
    if a.cmd == "train":
        _, info = train(a.n_train, a.epochs, a.lr, out=a.out, spec=spec)
        print(json.dumps(info))
    else:
        print(json.dumps(evaluate(a.weights, a.seeds, spec=spec)))


if __name__ == "__main__":
    main()
