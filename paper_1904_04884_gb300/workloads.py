"""Named synthetic workloads shaped like the paper's reconstructions.

The paper's own data (a turbulence database, experimental holograms) is not
available, so these seeded particle fields stand in for it. Shapes and optics
follow the paper's cases: 512x512 holograms with hundreds of planes at 10 um /
632 nm (Section 3.2), 1024x1024 at 532 nm with a few hundred planes
(Section 3.3). Where a workload leaves a value open the choice is stated here.

Each workload gives the opacity volume (via ``synth``) and the solver settings.
The hologram is formed by the caller's forward operator.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import synth


@dataclass(frozen=True)
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    wavelength: float        # metres
    pitch: float             # metres
    z0: float                # metres
    dz: float                # metres
    n_discs: int
    d_um: tuple              # (lo, hi) disc diameter in um
    at_voxel_centres: bool
    sigma: float             # hologram noise std
    iters: int
    lam_l1: float
    lam_tv: float
    n_inner: int             # TV dual gradient-projection steps per prox
    n_fibres: int = 0
    fibre_len_um: tuple = (50.0, 200.0)
    fibre_width_um: float = 3.0
    seed: int = 0
    tv_dims: int = 3
    z_slab: tuple = ()       # (lo, hi): discs only on planes lo..hi-1; () = all planes
    extra: dict = field(default_factory=dict)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def nvox(self):
        return self.nx * self.ny * self.nz

    def optics_tuple(self):
        return (self.nx, self.ny, self.nz, self.wavelength, self.pitch, self.z0, self.dz)

    def _draw_discs(self, st: "synth.Stream") -> "synth.Particles":
        lo, hi = self.z_slab or (0, self.nz)
        parts = synth.random_discs(st, (hi - lo, self.ny, self.nx), self.n_discs,
                                   self.d_um[0], self.d_um[1], self.pitch * 1e6,
                                   self.at_voxel_centres)
        parts.z += lo
        return parts

    def discs(self) -> "synth.Particles":
        """The placed discs (the same draws ``opacity`` rasterises)."""
        return self._draw_discs(synth.Stream(self.seed))

    def opacity(self) -> np.ndarray:
        """The seeded opacity volume a (float32 [nz][ny][nx])."""
        st = synth.Stream(self.seed)
        vol = np.zeros(self.shape, np.float32)
        synth.rasterise_discs(vol, self._draw_discs(st))
        if self.n_fibres:
            synth.rasterise_fibres(vol, st, self.n_fibres, self.fibre_len_um[0],
                                   self.fibre_len_um[1], self.fibre_width_um,
                                   self.pitch * 1e6, self.dz * 1e6)
        return vol

    def noise(self) -> np.ndarray:
        """Standard-normal hologram noise (float64 [ny][nx]), its own stream."""
        return synth.Stream(self.seed + 0x5EED).normal(self.nx * self.ny).reshape(self.ny, self.nx)


# 64x64 hologram, 16 planes; 20 discs of 30 um at voxel centres.
TINY = Workload("fista_tiny_64x64x16", 64, 64, 16, 632.8e-9, 10e-6, 5e-3, 100e-6,
                n_discs=20, d_um=(30.0, 30.0), at_voxel_centres=True, sigma=0.01,
                iters=50, lam_l1=0.01, lam_tv=0.005, n_inner=20)

# 512x512 hologram, 128 planes; 2,000 discs of 10-20 um. Regularisation weights
# are not given for this size; the tiny case's values are reused.
MID = Workload("fista_mid_512x512x128", 512, 512, 128, 532e-9, 5e-6, 5e-3, 50e-6,
               n_discs=2000, d_um=(10.0, 20.0), at_voxel_centres=False, sigma=0.02,
               iters=200, lam_l1=0.01, lam_tv=0.005, n_inner=20)

# 1024x1024 hologram, 256 planes; 10,000 discs of 8 um and 200 fibres.
LARGE = Workload("fista_large_1024x1024x256", 1024, 1024, 256, 532e-9, 5e-6, 5e-3, 25e-6,
                 n_discs=10000, d_um=(8.0, 8.0), at_voxel_centres=False, sigma=0.02,
                 iters=300, lam_l1=0.01, lam_tv=0.005, n_inner=20, n_fibres=200)

# The paper's turbulence case shape for context: 512x512x700 at 10 um / 632 nm,
# lam_l1 = 0.5, lam_FL = 0.2, 100 iterations (Section 3.2).
PAPER_TURBULENCE = Workload("paper_turbulence_512x512x700", 512, 512, 700, 632e-9, 10e-6,
                            5e-3, 10e-6, n_discs=5000, d_um=(10.0, 10.0),
                            at_voxel_centres=False, sigma=0.02, iters=100, lam_l1=0.5,
                            lam_tv=0.2, n_inner=20)

# A thin particle layer inside a deeper reconstructed volume: 1,000 discs of
# 10-20 um on planes 96-159 of 256 (a 3.2 mm layer in 12.8 mm of depth), with
# the plane-wise TV, weights and 5 gradient-projection steps of the paper's
# cuvette case (Section 3.3). Planes far from the layer can end up all zero,
# which the forward propagation then skips.
SLAB = Workload("slab_512x512x256", 512, 512, 256, 532e-9, 5e-6, 5e-3, 50e-6,
                n_discs=1000, d_um=(10.0, 20.0), at_voxel_centres=False, sigma=0.02,
                iters=100, lam_l1=0.1, lam_tv=0.1, n_inner=5, tv_dims=2, z_slab=(96, 160))

# The paper's 10^9-voxel example (Sections 1 and 2: 1024 x 1024 pixels and
# 1024 planes, 1,000 particles per hologram): 25 um planes at the large
# workload's optics, discs of 8-20 um, the paper's turbulence-case weights
# (its example names none), 100 iterations.
GIGA = Workload("fista_giga_1024x1024x1024", 1024, 1024, 1024, 532e-9, 5e-6, 5e-3, 25e-6,
                n_discs=1000, d_um=(8.0, 20.0), at_voxel_centres=False, sigma=0.02,
                iters=100, lam_l1=0.5, lam_tv=0.2, n_inner=20)

ALL = {w.name: w for w in (TINY, MID, LARGE, PAPER_TURBULENCE, SLAB, GIGA)}


def shadow_density(n_per_volume: float, depth: float, diameter: float, area: float) -> float:
    """Shadow density s_d = n_s L d^2 (Section 1, Eq. shadow_density), with the
    number concentration n_s = n / (area * depth)."""
    n_s = n_per_volume / (area * depth)
    return n_s * depth * diameter ** 2
