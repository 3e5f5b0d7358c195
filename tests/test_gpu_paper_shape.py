"""Parity at the paper's turbulence reconstruction size, 512 x 512 x 700
planes at 10 um (Section 3.2), on outputs the oracle can compute one by one:
the forward model of a volume with three non-zero planes (the oracle's
forward of each one-plane slab, summed), three planes of the adjoint, the
adjoint identity over the whole volume, and the fused-lasso prox at the
paper's K = 20 and at an odd K on crops whose interior the crop boundary does
not reach."""
import dataclasses

import numpy as np
import pytest
import torch

from oracle import rihv_oracle as O
from paper_1904_04884_gb300 import synth, workloads
from paper_1904_04884_gb300.rihv import Rihv

pytestmark = pytest.mark.gpu

OP_TOL = 1e-5
W = workloads.PAPER_TURBULENCE


def rel_l2(a, b):
    a = np.asarray(a, np.complex128)
    b = np.asarray(b, np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def slab(op, j):
    return dataclasses.replace(op, nz=1, z0=op.z0 + j * op.dz)


@pytest.fixture(scope="module")
def paper():
    assert torch.cuda.is_available()
    op = O.Optics(*W.optics_tuple())
    return op, Rihv(*W.optics_tuple())


def test_forward_of_sparse_planes(paper):
    op, h = paper
    dev = torch.device("cuda:0")
    x = torch.zeros(op.shape, dtype=torch.complex64, device=dev)
    ref = np.zeros((op.ny, op.nx), np.complex128)
    for n, j in enumerate((0, 351, 699)):
        p = synth.random_complex(synth.Stream(700 + n), (1, op.ny, op.nx)).astype(np.complex64)
        x[j] = torch.from_numpy(p[0]).to(dev)
        ref += O.forward(p.astype(np.complex128), slab(op, j))
    out = torch.empty((op.ny, op.nx), dtype=torch.complex64, device=dev)
    h.forward(x, out)
    torch.cuda.synchronize()
    assert rel_l2(out.cpu().numpy(), ref) <= OP_TOL


def test_adjoint_planes_and_identity(paper):
    op, h = paper
    dev = torch.device("cuda:0")
    r = synth.random_complex(synth.Stream(710), (op.ny, op.nx)).astype(np.complex64)
    vol = torch.empty(op.shape, dtype=torch.complex64, device=dev)
    h.adjoint(torch.from_numpy(r).to(dev), vol)
    torch.cuda.synchronize()
    for j in (0, 350, 699):
        ref = O.adjoint(r.astype(np.complex128), slab(op, j))[0]
        assert rel_l2(vol[j].cpu().numpy(), ref) <= OP_TOL, j
    blk = synth.random_complex(synth.Stream(711), (7, op.ny, op.nx)).astype(np.complex64)
    x = torch.from_numpy(blk).to(dev).repeat(op.nz // 7, 1, 1)
    hx = torch.empty((op.ny, op.nx), dtype=torch.complex64, device=dev)
    h.forward(x, hx)
    rt = torch.from_numpy(r).to(dev)
    lhs = torch.vdot(rt.flatten().to(torch.complex128), hx.flatten().to(torch.complex128))
    rhs = torch.vdot(vol.flatten().to(torch.complex128), x.flatten().to(torch.complex128))
    scale = (torch.linalg.vector_norm(hx.to(torch.complex128)) *
             torch.linalg.vector_norm(rt.to(torch.complex128)))
    assert abs(complex(lhs - rhs)) / float(scale) < 1e-5


@pytest.mark.parametrize("dims", [3, 2])
@pytest.mark.parametrize("k", [20, 5])
def test_prox_on_crops(paper, k, dims):
    """v is a seeded 28 x 64 x 64 block tiled over the volume (700 = 25 x 28).
    The prox at a voxel depends on v within k + 1 voxels, so on a crop with a
    margin of k + 2 (none at the volume's own faces) the oracle's prox of the
    crop equals the full-size result."""
    op, h = paper
    dev = torch.device("cuda:0")
    blk = synth.random_complex(synth.Stream(720), (28, 64, 64)).astype(np.complex64)
    v = torch.from_numpy(blk).to(dev).repeat(op.nz // 28, op.ny // 64, op.nx // 64)
    out = torch.empty_like(v)
    t_l1, t_tv = 0.3, 0.05
    h.set_options(tv_dims=dims)
    h.prox_fused_lasso(v, t_l1, t_tv, k, out)
    torch.cuda.synchronize()
    m = k + 2
    size = 2 * m + 12
    for (z0, y0, x0) in ((0, 0, 0), (333, 200, 250), (700 - size, 512 - size, 512 - size)):
        z1, y1, x1 = z0 + size, y0 + size, x0 + size
        crop = blk[np.ix_(np.arange(z0, z1) % 28, np.arange(y0, y1) % 64,
                          np.arange(x0, x1) % 64)].astype(np.complex128)
        ref = O.prox_fused_lasso(crop, t_l1, t_tv, k, dims)
        got = out[z0:z1, y0:y1, x0:x1].cpu().numpy()
        sl = tuple(slice(m if a > 0 else 0, (b - a) - (m if b < n else 0))
                   for a, b, n in ((z0, z1, op.nz), (y0, y1, op.ny), (x0, x1, op.nx)))
        assert rel_l2(got[sl], ref[sl]) <= OP_TOL, (z0, y0, x0)
