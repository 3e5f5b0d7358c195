"""Seeded synthetic inputs: particle volumes, fibres, vortex advection, noise.

This module holds no reconstruction arithmetic: no transfer function, no FFT,
no prox. It draws random numbers and rasterises objects. Holograms are formed
by the caller, who applies its own forward operator to the volume this module
returns and then calls ``intensity_hologram`` or ``linear_hologram`` with the
modelled field and a noise field drawn here.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): a counter-based generator, so
draw n of a stream is mix(seed + (n + 1) * gamma) and any range of draws can be
produced without the ones before it. Uniform doubles take the top 53 bits;
normals use the Box-Muller transform on pairs of uniforms.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, start: int, n: int) -> np.ndarray:
    """Draws start .. start+n-1 of the SplitMix64 stream for ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        ctr = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + ctr * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


class Stream:
    """A sequential view of one SplitMix64 stream."""

    def __init__(self, seed: int):
        self.seed = int(seed)
        self.count = 0

    def bits(self, n: int) -> np.ndarray:
        out = splitmix64(self.seed, self.count, n)
        self.count += n
        return out

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        """n doubles in [lo, hi) from the top 53 bits of each draw."""
        u = (self.bits(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        return lo + (hi - lo) * u

    def integers(self, n: int, hi: int) -> np.ndarray:
        """n integers in [0, hi) (floor of a uniform; bias < 2^-40 for hi < 2^13)."""
        return np.minimum(np.floor(self.uniform(n) * hi).astype(np.int64), hi - 1)

    def normal(self, n: int) -> np.ndarray:
        """n standard normals by Box-Muller on ceil(n/2) pairs of uniforms."""
        m = (n + 1) // 2
        u1 = self.uniform(m)
        u2 = self.uniform(m)
        r = np.sqrt(-2.0 * np.log1p(-u1))          # 1 - u1 is in (0, 1]
        th = 2.0 * np.pi * u2
        out = np.empty(2 * m)
        out[0::2] = r * np.cos(th)
        out[1::2] = r * np.sin(th)
        return out[:n]


# --------------------------------------------------------------------------
# Object rasterisation
# --------------------------------------------------------------------------

@dataclass
class Particles:
    """Disc particles: centres in voxel units (x, y continuous, z a plane index)
    and diameters in pixels."""
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    d_px: np.ndarray

    def __len__(self):
        return len(self.x)


def random_discs(stream: Stream, shape, n: int, d_um_lo: float, d_um_hi: float,
                 pitch_um: float, at_voxel_centres: bool) -> Particles:
    """n discs with uniform random position and uniform diameter in [lo, hi] um."""
    nz, ny, nx = shape
    if at_voxel_centres:
        x = stream.integers(n, nx) + 0.5
        y = stream.integers(n, ny) + 0.5
    else:
        x = stream.uniform(n, 0.0, nx)
        y = stream.uniform(n, 0.0, ny)
    z = stream.integers(n, nz)
    d = stream.uniform(n, d_um_lo, d_um_hi) if d_um_hi > d_um_lo else np.full(n, d_um_lo)
    return Particles(x.astype(np.float64), y.astype(np.float64), z.astype(np.int64),
                     d / pitch_um)


def rasterise_discs(vol: np.ndarray, parts: Particles, supersample: int = 4) -> None:
    """Adds opaque in-plane discs to ``vol`` ([nz][ny][nx] float) in place.

    Pixel i covers [i, i+1); its value is the fraction of an s x s grid of
    sample points inside the disc. Overlaps keep the larger value.
    """
    nz, ny, nx = vol.shape
    s = supersample
    offs = (np.arange(s) + 0.5) / s
    for cx, cy, cz, dpx in zip(parts.x, parts.y, parts.z, parts.d_px):
        r = 0.5 * dpx
        i0 = max(int(math.floor(cx - r)), 0)
        i1 = min(int(math.ceil(cx + r)), nx)
        j0 = max(int(math.floor(cy - r)), 0)
        j1 = min(int(math.ceil(cy + r)), ny)
        if i1 <= i0 or j1 <= j0:
            continue
        sx = (np.arange(i0, i1)[:, None] + offs[None, :]).ravel()
        sy = (np.arange(j0, j1)[:, None] + offs[None, :]).ravel()
        inside = ((sy[:, None] - cy) ** 2 + (sx[None, :] - cx) ** 2) <= r * r
        cov = inside.reshape(j1 - j0, s, i1 - i0, s).mean(axis=(1, 3))
        sub = vol[int(cz), j0:j1, i0:i1]
        np.maximum(sub, cov, out=sub)


def rasterise_fibres(vol: np.ndarray, stream: Stream, n: int, len_um_lo: float,
                     len_um_hi: float, width_um: float, pitch_um: float,
                     dz_um: float) -> None:
    """Adds n straight opaque fibres (isotropic orientation) to ``vol`` in place.

    A voxel whose centre lies within max(width/2, pitch/2) of the fibre axis
    segment (physical distance) is set to 1.
    """
    nz, ny, nx = vol.shape
    cx = stream.uniform(n, 0.0, nx * pitch_um)
    cy = stream.uniform(n, 0.0, ny * pitch_um)
    cz = stream.uniform(n, 0.0, nz * dz_um)
    length = stream.uniform(n, len_um_lo, len_um_hi)
    cos_t = stream.uniform(n, -1.0, 1.0)
    phi = stream.uniform(n, 0.0, 2.0 * np.pi)
    sin_t = np.sqrt(1.0 - cos_t ** 2)
    ux, uy, uz = sin_t * np.cos(phi), sin_t * np.sin(phi), cos_t
    rad = max(0.5 * width_um, 0.5 * pitch_um)
    for f in range(n):
        half = 0.5 * length[f]
        p0 = np.array([cx[f] - half * ux[f], cy[f] - half * uy[f], cz[f] - half * uz[f]])
        p1 = np.array([cx[f] + half * ux[f], cy[f] + half * uy[f], cz[f] + half * uz[f]])
        lo = np.minimum(p0, p1) - rad
        hi = np.maximum(p0, p1) + rad
        i0, i1 = max(int(lo[0] // pitch_um), 0), min(int(hi[0] // pitch_um) + 1, nx)
        j0, j1 = max(int(lo[1] // pitch_um), 0), min(int(hi[1] // pitch_um) + 1, ny)
        k0, k1 = max(int(lo[2] // dz_um), 0), min(int(hi[2] // dz_um) + 1, nz)
        if i1 <= i0 or j1 <= j0 or k1 <= k0:
            continue
        kk, jj, ii = np.meshgrid(np.arange(k0, k1), np.arange(j0, j1), np.arange(i0, i1),
                                 indexing="ij")
        px = (ii + 0.5) * pitch_um
        py = (jj + 0.5) * pitch_um
        pz = (kk + 0.5) * dz_um
        d = p1 - p0
        seg2 = float(d @ d)
        t = ((px - p0[0]) * d[0] + (py - p0[1]) * d[1] + (pz - p0[2]) * d[2]) / seg2
        t = np.clip(t, 0.0, 1.0)
        dist2 = ((px - p0[0] - t * d[0]) ** 2 + (py - p0[1] - t * d[1]) ** 2
                 + (pz - p0[2] - t * d[2]) ** 2)
        sub = vol[k0:k1, j0:j1, i0:i1]
        sub[dist2 <= rad * rad] = 1.0


def lamb_oseen_advect(x: np.ndarray, y: np.ndarray, gamma: float, r_core: float,
                      cx: float, cy: float, frames: float = 1.0, substeps: int = 4):
    """Advects points by a Lamb-Oseen vortex (axis along z through (cx, cy)).

    Azimuthal speed u(r) = gamma / (2 pi r) * (1 - exp(-r^2 / r_core^2)); classic
    fourth-order Runge-Kutta over ``frames`` time units in ``substeps`` steps.
    Units: pixels and frames.
    """
    def vel(px, py):
        dx, dy = px - cx, py - cy
        r2 = dx * dx + dy * dy
        with np.errstate(divide="ignore", invalid="ignore"):
            f = np.where(r2 > 0, gamma / (2.0 * np.pi * r2) * (-np.expm1(-r2 / r_core ** 2)),
                         gamma / (2.0 * np.pi * r_core ** 2))
        return -f * dy, f * dx

    h = frames / substeps
    for _ in range(substeps):
        k1x, k1y = vel(x, y)
        k2x, k2y = vel(x + 0.5 * h * k1x, y + 0.5 * h * k1y)
        k3x, k3y = vel(x + 0.5 * h * k2x, y + 0.5 * h * k2y)
        k4x, k4y = vel(x + h * k3x, y + h * k3y)
        x = x + h / 6.0 * (k1x + 2 * k2x + 2 * k3x + k4x)
        y = y + h / 6.0 * (k1y + 2 * k2y + 2 * k3y + k4y)
    return x, y


# --------------------------------------------------------------------------
# Hologram formation from a modelled field (the caller applies its own H)
# --------------------------------------------------------------------------

def intensity_hologram(field: np.ndarray, sigma: float, noise: np.ndarray) -> np.ndarray:
    """Recorded contrast hologram b = 1 - |1 - field|^2 + sigma * noise (float32).

    ``field`` is the modelled scattered field H a of an opacity volume a; its
    linearisation is b ~ 2 Re(H a).
    """
    b = 1.0 - np.abs(1.0 - field) ** 2 + sigma * noise.reshape(field.shape)
    return b.astype(np.float32)


def linear_hologram(field: np.ndarray, sigma: float, noise: np.ndarray) -> np.ndarray:
    """Linear test hologram b = Re(field) + sigma * noise (float32)."""
    return (field.real + sigma * noise.reshape(field.shape)).astype(np.float32)


def random_complex(stream: Stream, shape) -> np.ndarray:
    """Complex array with independent standard-normal real and imaginary parts."""
    n = int(np.prod(shape))
    g = stream.normal(2 * n)
    return (g[0::2] + 1j * g[1::2]).reshape(shape)
