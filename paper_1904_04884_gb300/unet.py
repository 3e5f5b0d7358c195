"""Learned warm start for FISTA: a small 3D U-Net on tcgen05 convolutions.

Not in the paper. The network maps the back-propagated hologram H^H b (two
channels: real and imaginary part) of one volume to an initial volume for the
fused-lasso FISTA solve, x0 = base_coeff * H^H b + scale_out * net(H^H b): the
first term is FISTA's own first iterate from zero (base_coeff = 2 tau), so the
network learns the correction that FISTA would otherwise build over many
iterations. Plain FISTA from zero remains the fallback and the reference for the
result (the solver refines x0 to the same objective).

Architecture (3 levels, 16/32/64 channels, 3x3x3 convolutions, BF16 weights
and activations, FP32 accumulation):

    level 1 (d, h, w)       : conv 16->16, conv 16->16 (skip s1)
    level 2 (d/2, h/2, w/2) : pool, conv 16->32, conv 32->32 (skip s2)
    level 3 (d/4, h/4, w/4) : pool, conv 32->64, conv 64->64
    level 2                 : upsample, concat s2 (96), conv 96->32, conv 32->32
    level 1                 : upsample, concat s1 (48), conv 48->16, conv 16->16,
                              conv 16->16 (output, no ReLU; channels 0, 1 used)

The input's two channels are zero-padded to 16 (the convolution kernels take
multiples of 16 channels), as are the output's. Every layer runs in librihv's
kernels (rihv_nn.h); this module allocates the tensors (PyTorch) and sequences
the calls. Parameters are FP32 masters with BF16 copies, trained with Adam.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import nn

LAYERS = [("e1a", 16, 16, True), ("e1b", 16, 16, True), ("e2a", 16, 32, True),
          ("e2b", 32, 32, True), ("b1", 32, 64, True), ("b2", 64, 64, True),
          ("d2a", 96, 32, True), ("d2b", 32, 32, True), ("d1a", 48, 16, True),
          ("d1b", 16, 16, True), ("out", 16, 16, False)]
REAL_IN = {"e1a": 2}            # input channels that carry data
REAL_OUT = {"out": 2}
C_IO = 16


class WarmStartUNet:
    def __init__(self, dims, seed=0, device="cuda:0"):
        d, h, w = dims
        if d % 4 or h % 4 or w % 4:
            raise ValueError("volume sizes must be multiples of 4")
        self.dev = torch.device(device)
        self.dims = [(d, h, w), (d // 2, h // 2, w // 2), (d // 4, h // 4, w // 4)]
        self.nv = [a * b * c for a, b, c in self.dims]
        g = torch.Generator().manual_seed(seed)
        self.W, self.Wb, self.b, self.gW, self.gb = {}, {}, {}, {}, {}
        self.m, self.v = {}, {}
        for name, cin, cout, _ in LAYERS:
            fan_in = 27 * REAL_IN.get(name, cin)
            w0 = torch.randn(cout, 27, cin, generator=g) * math.sqrt(2.0 / fan_in)
            if name in REAL_IN:
                w0[:, :, REAL_IN[name]:] = 0
            if name == "out":
                w0 *= 0.1
                w0[REAL_OUT[name]:] = 0
            self._set(name, w0, torch.zeros(cout))
        self.scale_in = 1.0
        self.scale_out = 1.0
        self.base_coeff = 0.0
        self.step_count = 0
        self.err = torch.zeros(1, dtype=torch.int32, device=self.dev)
        self._bufs = {}

    def _set(self, name, w, b):
        self.W[name] = w.to(self.dev, torch.float32).contiguous()
        self.Wb[name] = self.W[name].to(torch.bfloat16).contiguous()
        self.b[name] = b.to(self.dev, torch.float32).contiguous()
        self.gW[name] = torch.zeros_like(self.W[name])
        self.gb[name] = torch.zeros_like(self.b[name])
        self.m[name] = (torch.zeros_like(self.W[name]), torch.zeros_like(self.b[name]))
        self.v[name] = (torch.zeros_like(self.W[name]), torch.zeros_like(self.b[name]))

    # ---- buffers ----------------------------------------------------------
    def _buf(self, key, level, c, dtype=torch.bfloat16):
        t = self._bufs.get(key)
        if t is None:
            t = torch.empty((self.nv[level], c), dtype=dtype, device=self.dev)
            self._bufs[key] = t
        return t

    def _conv(self, name, x, level, out):
        _, cin, cout, relu = next(l for l in LAYERS if l[0] == name)
        nn.conv3d(x, self.Wb[name], self.b[name], out, self.dims[level], cin, cout, relu, self.err)
        return out

    # ---- forward ----------------------------------------------------------
    def forward(self, inp):
        """inp: BF16 [voxels][16] at level 1. Returns FP32 [voxels][16]."""
        B = self._buf
        a = {"x0": inp}
        a["e1a"] = self._conv("e1a", inp, 0, B("e1a", 0, 16))
        a["s1"] = self._conv("e1b", a["e1a"], 0, B("s1", 0, 16))
        a["p1"] = B("p1", 1, 16)
        nn.avgpool2(a["s1"], a["p1"], self.dims[0], 16)
        a["e2a"] = self._conv("e2a", a["p1"], 1, B("e2a", 1, 32))
        a["s2"] = self._conv("e2b", a["e2a"], 1, B("s2", 1, 32))
        a["p2"] = B("p2", 2, 32)
        nn.avgpool2(a["s2"], a["p2"], self.dims[1], 32)
        a["b1"] = self._conv("b1", a["p2"], 2, B("b1", 2, 64))
        a["b2"] = self._conv("b2", a["b1"], 2, B("b2", 2, 64))
        u2 = B("u2", 1, 64)
        nn.upsample2(a["b2"], u2, self.dims[2], 64)
        a["c2"] = B("c2", 1, 96)
        nn.concat(u2, a["s2"], a["c2"], self.nv[1], 64, 32)
        a["d2a"] = self._conv("d2a", a["c2"], 1, B("d2a", 1, 32))
        a["d2b"] = self._conv("d2b", a["d2a"], 1, B("d2b", 1, 32))
        u1 = B("u1", 0, 32)
        nn.upsample2(a["d2b"], u1, self.dims[1], 32)
        a["c1"] = B("c1", 0, 48)
        nn.concat(u1, a["s1"], a["c1"], self.nv[0], 32, 16)
        a["d1a"] = self._conv("d1a", a["c1"], 0, B("d1a", 0, 16))
        a["d1b"] = self._conv("d1b", a["d1a"], 0, B("d1b", 0, 16))
        out = self._conv("out", a["d1b"], 0, B("out", 0, 16, torch.float32))
        self.acts = a
        return out

    # ---- backward ---------------------------------------------------------
    def _layer_back(self, name, x_in, level, g, y_out=None, need_dgrad=True):
        """g: BF16 gradient at the layer's output (after ReLU). Fills gW, gb and
        returns the BF16 gradient at its input."""
        _, cin, cout, relu = next(l for l in LAYERS if l[0] == name)
        if relu:
            gr = self._buf(f"gr_{level}_{cout}", level, cout)
            nn.relu_grad(g, y_out, gr)
            g = gr
        dims = self.dims[level]
        work = self._bufs.get("wg_work")
        need = nn.wgrad_workspace_bytes(dims, cin, cout)
        if work is None or work.numel() * 4 < need:
            work = torch.empty(need // 4 + 64, dtype=torch.float32, device=self.dev)
            self._bufs["wg_work"] = work
        nn.conv3d_wgrad(x_in, g, self.gW[name], dims, cin, cout, work, self.err)
        bw = self._bufs.get("bg_work")
        if bw is None:
            bw = torch.empty(256 * 128, dtype=torch.float64, device=self.dev)
            self._bufs["bg_work"] = bw
        nn.bias_grad(g, self.gb[name], self.nv[level], cout, bw)
        if not need_dgrad:
            return None
        gx = self._buf(f"gx_{name}", level, cin)
        nn.conv3d_dgrad(g, self.Wb[name], gx, dims, cin, cout, self.err)
        return gx

    def backward(self, g_out):
        a = self.acts
        B = self._buf
        g = self._layer_back("out", a["d1b"], 0, g_out)
        g = self._layer_back("d1b", a["d1a"], 0, g, a["d1b"])
        g = self._layer_back("d1a", a["c1"], 0, g, a["d1a"])
        gu1, gs1 = B("gu1", 0, 32), B("gs1", 0, 16)
        nn.split(g, gu1, gs1, self.nv[0], 32, 16)
        g = B("gup1", 1, 32)
        nn.upsample2_grad(gu1, g, self.dims[1], 32)
        g = self._layer_back("d2b", a["d2a"], 1, g, a["d2b"])
        g = self._layer_back("d2a", a["c2"], 1, g, a["d2a"])
        gu2, gs2 = B("gu2", 1, 64), B("gs2", 1, 32)
        nn.split(g, gu2, gs2, self.nv[1], 64, 32)
        g = B("gup2", 2, 64)
        nn.upsample2_grad(gu2, g, self.dims[2], 64)
        g = self._layer_back("b2", a["b1"], 2, g, a["b2"])
        g = self._layer_back("b1", a["p2"], 2, g, a["b1"])
        gp = B("gpool2", 1, 32)
        nn.avgpool2_grad(g, gp, self.dims[1], 32)
        nn.add(gp, gs2, gp)
        g = self._layer_back("e2b", a["e2a"], 1, gp, a["s2"])
        g = self._layer_back("e2a", a["p1"], 1, g, a["e2a"])
        gp = B("gpool1", 0, 16)
        nn.avgpool2_grad(g, gp, self.dims[0], 16)
        nn.add(gp, gs1, gp)
        g = self._layer_back("e1b", a["e1a"], 0, gp, a["s1"])
        self._layer_back("e1a", a["x0"], 0, g, a["e1a"], need_dgrad=False)

    def adam_step(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.step_count += 1
        for name, *_ in LAYERS:
            mw, mb = self.m[name]
            vw, vb = self.v[name]
            nn.adam(self.W[name], self.gW[name], mw, vw, self.Wb[name], lr, beta1, beta2, eps,
                    self.step_count)
            bb = self._bufs.get(f"bias_bf16_{name}")
            if bb is None:
                bb = torch.empty_like(self.b[name], dtype=torch.bfloat16)
                self._bufs[f"bias_bf16_{name}"] = bb
            nn.adam(self.b[name], self.gb[name], mb, vb, bb, lr, beta1, beta2, eps,
                    self.step_count)

    # ---- training / inference helpers ---------------------------------------
    def pack(self, hb):
        """Network input from the complex back-propagated hologram [d][h][w]."""
        inp = self._buf("inp", 0, C_IO)
        nn.pack_input(hb, inp, self.nv[0], C_IO, self.scale_in)
        return inp

    def train_step(self, hb, target, lr=1e-3):
        """One Adam step on MSE(net(hb), target / scale_out); returns the loss.
        target is the correction x* - base_coeff * hb."""
        out = self.forward(self.pack(hb))
        g = self._buf("gout", 0, C_IO)
        loss = self._bufs.get("loss")
        if loss is None:
            loss = torch.zeros(1, dtype=torch.float64, device=self.dev)
            self._bufs["loss"] = loss
            self._bufs["mse_work"] = torch.empty(1024, dtype=torch.float64, device=self.dev)
        nn.mse_grad(out, target, g, loss, self.nv[0], C_IO, self.scale_out, self._bufs["mse_work"])
        self.backward(g)
        self.adam_step(lr)
        return loss

    def predict(self, hb, x0_out):
        """x0 = base_coeff * H^H b + scale_out * net(scale_in * H^H b)."""
        out = self.forward(self.pack(hb))
        nn.unpack_output(out, x0_out, self.nv[0], C_IO, self.scale_out, base=hb,
                         base_scale=self.base_coeff)
        return x0_out

    def state(self):
        st = {f"W_{n}": self.W[n].cpu().numpy() for n, *_ in LAYERS}
        st.update({f"b_{n}": self.b[n].cpu().numpy() for n, *_ in LAYERS})
        st["scale_in"] = np.float64(self.scale_in)
        st["scale_out"] = np.float64(self.scale_out)
        st["base_coeff"] = np.float64(self.base_coeff)
        st["dims"] = np.array(self.dims[0])
        return st

    def save(self, path):
        np.savez(path, **self.state())

    @classmethod
    def load(cls, path, device="cuda:0"):
        st = np.load(path)
        net = cls(tuple(int(v) for v in st["dims"]), device=device)
        for n, *_ in LAYERS:
            net._set(n, torch.from_numpy(st[f"W_{n}"]), torch.from_numpy(st[f"b_{n}"]))
        net.scale_in = float(st["scale_in"])
        net.scale_out = float(st["scale_out"])
        net.base_coeff = float(st["base_coeff"]) if "base_coeff" in st else 0.0
        return net

    def errors(self):
        return int(self.err.item())
