"""FP64 CPU oracle for the warm-start network's layers.

TEST INFRASTRUCTURE ONLY (same rules as rihv_oracle: only tests, smoke() and
bench.py's CPU legs use it; it imports nothing from the product package).

The network is not in the paper; it is the project's learned warm start for
FISTA. Layers, with activations in N D H W C order (one sample, channels
last) and weights W[c_out][tap][c_in] with tap = (dz+1)*9 + (dy+1)*3 + (dx+1):

- conv3d (3x3x3, stride 1, zero padding 1): y[v, o] = b[o] + sum_{t, c} W[o, t, c] x[v + off_t, c]
- its input gradient (dgrad) and weight gradient (wgrad), written out from
  the definition (sums over shifted copies), not from the forward code
- 2x2x2 average pooling and nearest-neighbour 2x upsampling, and their
  adjoints; ReLU.
"""
from __future__ import annotations

import numpy as np

OFFSETS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def _shift(x, dz, dy, dx):
    """s[z, y, x] = x[z + dz, y + dy, x + dx], zero outside (x is [D][H][W][C])."""
    d, h, w = x.shape[:3]
    out = np.zeros_like(x)
    zs, ze = max(0, -dz), min(d, d - dz)
    ys, ye = max(0, -dy), min(h, h - dy)
    xs, xe = max(0, -dx), min(w, w - dx)
    out[zs:ze, ys:ye, xs:xe] = x[zs + dz:ze + dz, ys + dy:ye + dy, xs + dx:xe + dx]
    return out


def conv3d(x, w, b=None):
    """x [D][H][W][Cin], w [Cout][27][Cin], b [Cout] -> [D][H][W][Cout] (FP64)."""
    x = np.asarray(x, np.float64)
    w = np.asarray(w, np.float64)
    y = np.zeros(x.shape[:3] + (w.shape[0],))
    for t, (dz, dy, dx) in enumerate(OFFSETS):
        y += _shift(x, dz, dy, dx) @ w[:, t, :].T
    if b is not None:
        y += np.asarray(b, np.float64)
    return y


def conv3d_dgrad(gy, w):
    """Gradient of sum(gy * conv3d(x, w)) with respect to x:
    gx[u, c] = sum_{t, o} W[o, t, c] gy[u - off_t, o]."""
    gy = np.asarray(gy, np.float64)
    w = np.asarray(w, np.float64)
    gx = np.zeros(gy.shape[:3] + (w.shape[2],))
    for t, (dz, dy, dx) in enumerate(OFFSETS):
        gx += _shift(gy, -dz, -dy, -dx) @ w[:, t, :]
    return gx


def conv3d_wgrad(x, gy):
    """Gradient with respect to W: gW[o, t, c] = sum_v gy[v, o] x[v + off_t, c]."""
    x = np.asarray(x, np.float64)
    gy = np.asarray(gy, np.float64)
    cin, cout = x.shape[3], gy.shape[3]
    gw = np.zeros((cout, 27, cin))
    g2 = gy.reshape(-1, cout)
    for t, (dz, dy, dx) in enumerate(OFFSETS):
        gw[:, t, :] = g2.T @ _shift(x, dz, dy, dx).reshape(-1, cin)
    return gw


def avgpool2(x):
    """2x2x2 mean pooling (even sizes)."""
    d, h, w, c = x.shape
    return np.asarray(x, np.float64).reshape(d // 2, 2, h // 2, 2, w // 2, 2, c).mean(axis=(1, 3, 5))


def avgpool2_grad(gy):
    """Adjoint of avgpool2: each input voxel receives 1/8 of its cell's gradient."""
    return np.repeat(np.repeat(np.repeat(np.asarray(gy, np.float64), 2, 0), 2, 1), 2, 2) / 8.0


def upsample2(x):
    """Nearest-neighbour 2x upsampling."""
    return np.repeat(np.repeat(np.repeat(np.asarray(x, np.float64), 2, 0), 2, 1), 2, 2)


def upsample2_grad(gy):
    """Adjoint of upsample2: sum over each 2x2x2 cell."""
    d, h, w, c = gy.shape
    return np.asarray(gy, np.float64).reshape(d // 2, 2, h // 2, 2, w // 2, 2, c).sum(axis=(1, 3, 5))


def relu(x):
    return np.maximum(np.asarray(x, np.float64), 0.0)
