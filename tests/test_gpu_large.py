"""Parity at the full size of the 1024 x 1024 x 256 workload (25 um planes),
on outputs the oracle can compute one by one: the forward model of a volume
with three non-zero planes (the oracle's forward of each one-plane slab,
summed), three planes of the adjoint (the oracle's adjoint of one-plane
slabs), the adjoint identity over the whole volume, and the fused-lasso prox
(first, middle and fused-final TV launches) on crops whose interior is
unaffected by the crop boundary."""
import dataclasses

import numpy as np
import pytest
import torch

from oracle import rihv_oracle as O
from paper_1904_04884_gb300 import synth, workloads
from paper_1904_04884_gb300.rihv import Rihv

pytestmark = pytest.mark.gpu

OP_TOL = 1e-5
W = workloads.LARGE


def rel_l2(a, b):
    a = np.asarray(a, np.complex128)
    b = np.asarray(b, np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def slab(op, j):
    """The one-plane optics of plane j of `op`."""
    return dataclasses.replace(op, nz=1, z0=op.z0 + j * op.dz)


@pytest.fixture(scope="module")
def large():
    assert torch.cuda.is_available()
    op = O.Optics(*W.optics_tuple())
    return op, Rihv(*W.optics_tuple())


def test_large_forward_of_sparse_planes(large):
    op, h = large
    dev = torch.device("cuda:0")
    planes = {0: None, 117: None, 255: None}
    x = torch.zeros(op.shape, dtype=torch.complex64, device=dev)
    ref = np.zeros((op.ny, op.nx), np.complex128)
    for n, j in enumerate(planes):
        p = synth.random_complex(synth.Stream(300 + n), (1, op.ny, op.nx))
        x[j] = torch.from_numpy(p[0].astype(np.complex64)).to(dev)
        ref += O.forward(p.astype(np.complex64).astype(np.complex128), slab(op, j))
    out = torch.empty((op.ny, op.nx), dtype=torch.complex64, device=dev)
    h.forward(x, out)
    torch.cuda.synchronize()
    assert rel_l2(out.cpu().numpy(), ref) <= OP_TOL


def test_large_adjoint_planes_and_identity(large):
    op, h = large
    dev = torch.device("cuda:0")
    r = synth.random_complex(synth.Stream(310), (op.ny, op.nx)).astype(np.complex64)
    vol = torch.empty(op.shape, dtype=torch.complex64, device=dev)
    h.adjoint(torch.from_numpy(r).to(dev), vol)
    torch.cuda.synchronize()
    for j in (0, 100, 255):
        ref = O.adjoint(r.astype(np.complex128), slab(op, j))[0]
        assert rel_l2(vol[j].cpu().numpy(), ref) <= OP_TOL, j
    # <H x, r> = <x, H^H r> over the whole volume, x with random planes tiled
    blk = synth.random_complex(synth.Stream(311), (8, op.ny, op.nx)).astype(np.complex64)
    x = torch.from_numpy(blk).to(dev).repeat(op.nz // 8, 1, 1)
    hx = torch.empty((op.ny, op.nx), dtype=torch.complex64, device=dev)
    h.forward(x, hx)
    rt = torch.from_numpy(r).to(dev)
    lhs = torch.vdot(rt.flatten().to(torch.complex128), hx.flatten().to(torch.complex128))
    rhs = torch.vdot(vol.flatten().to(torch.complex128), x.flatten().to(torch.complex128))
    scale = (torch.linalg.vector_norm(hx.to(torch.complex128)) *
             torch.linalg.vector_norm(rt.to(torch.complex128)))
    assert abs(complex(lhs - rhs)) / float(scale) < 1e-5


@pytest.mark.parametrize("k", [4, 5])
def test_large_prox_on_crops(large, k):
    """v is a seeded 32 x 64 x 64 block tiled over the volume. The prox at a
    voxel depends on v within k + 1 voxels, so on a crop with an 8-voxel
    margin (none at the volume's own faces) the oracle's prox of the crop
    equals the full-size result. k = 4: first, then fused-final launch; k = 5:
    a single first step, one launch reading p, then the fused-final launch."""
    op, h = large
    dev = torch.device("cuda:0")
    blk = synth.random_complex(synth.Stream(320), (32, 64, 64)).astype(np.complex64)
    reps = (op.nz // 32, op.ny // 64, op.nx // 64)
    v = torch.from_numpy(blk).to(dev).repeat(*reps)
    out = torch.empty_like(v)
    t_l1, t_tv = 0.3, 0.05
    h.set_options(tv_dims=3)
    h.prox_fused_lasso(v, t_l1, t_tv, k, out)
    torch.cuda.synchronize()
    m = 8
    for (z0, y0, x0) in ((0, 0, 0), (100, 500, 300), (224, 984, 984)):
        z1, y1, x1 = min(op.nz, z0 + 32), min(op.ny, y0 + 40), min(op.nx, x0 + 40)
        # the same input on the host: the tiled block, indexed modulo its size
        crop = blk[np.ix_(np.arange(z0, z1) % 32, np.arange(y0, y1) % 64,
                          np.arange(x0, x1) % 64)].astype(np.complex128)
        ref = O.prox_fused_lasso(crop, t_l1, t_tv, k, 3)
        got = out[z0:z1, y0:y1, x0:x1].cpu().numpy()
        # interior: drop the margin on crop faces that are not volume faces
        sl = tuple(slice(m if a > 0 else 0, (b - a) - (m if b < n else 0))
                   for a, b, n in ((z0, z1, op.nz), (y0, y1, op.ny), (x0, x1, op.nx)))
        assert rel_l2(got[sl], ref[sl]) <= OP_TOL, (z0, y0, x0)
