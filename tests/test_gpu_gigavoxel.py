"""A 10^9-voxel reconstruction: the paper's 1024 x 1024 x 1024 example
(Sections 1 and 2) with its whole dense working state in HBM (about 90 GB).

Parity on outputs the oracle can compute one by one, as at 1024 x 1024 x 256:
the forward model of a volume with three non-zero planes, three planes of the
adjoint, the prox on crops whose interior the crop boundary does not reach,
and the first FISTA iterate x_1 = prox(2 tau H^H b) (the solver's own
gradient step and prox at this size) on a crop. Then a short sequence of
frames stored in per-plane COO form between frames: every stored form expands
to the frame's solution bit for bit, is much smaller than the dense volume,
gives the same detections, and warm-starts the next frame.
"""
import dataclasses

import numpy as np
import pytest
import torch

from oracle import rihv_oracle as O
from paper_1904_04884_gb300 import coo_sequence, synth, workloads
from paper_1904_04884_gb300.rihv import Rihv

pytestmark = pytest.mark.gpu

OP_TOL = 1e-5
W = workloads.GIGA


def rel_l2(a, b):
    a = np.asarray(a, np.complex128)
    b = np.asarray(b, np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def slab(op, j, n=1):
    """The optics of planes j .. j+n-1 of `op`."""
    return dataclasses.replace(op, nz=n, z0=op.z0 + j * op.dz)


@pytest.fixture(scope="module")
def giga():
    assert torch.cuda.is_available()
    op = O.Optics(*W.optics_tuple())
    h = Rihv(*W.optics_tuple())
    yield op, h
    h.close()
    torch.cuda.empty_cache()


def test_giga_forward_of_sparse_planes(giga):
    op, h = giga
    dev = torch.device("cuda:0")
    x = torch.zeros(op.shape, dtype=torch.complex64, device=dev)
    ref = np.zeros((op.ny, op.nx), np.complex128)
    for n, j in enumerate((0, 511, 1023)):
        p = synth.random_complex(synth.Stream(400 + n), (1, op.ny, op.nx)).astype(np.complex64)
        x[j] = torch.from_numpy(p[0]).to(dev)
        ref += O.forward(p.astype(np.complex128), slab(op, j))
    out = torch.empty((op.ny, op.nx), dtype=torch.complex64, device=dev)
    h.forward(x, out)
    torch.cuda.synchronize()
    del x
    assert rel_l2(out.cpu().numpy(), ref) <= OP_TOL


def test_giga_adjoint_planes(giga):
    op, h = giga
    dev = torch.device("cuda:0")
    r = synth.random_complex(synth.Stream(410), (op.ny, op.nx)).astype(np.complex64)
    vol = torch.empty(op.shape, dtype=torch.complex64, device=dev)
    h.adjoint(torch.from_numpy(r).to(dev), vol)
    torch.cuda.synchronize()
    for j in (0, 600, 1023):
        ref = O.adjoint(r.astype(np.complex128), slab(op, j))[0]
        assert rel_l2(vol[j].cpu().numpy(), ref) <= OP_TOL, j
    del vol


def test_giga_prox_on_crops(giga):
    """v is a seeded 32 x 64 x 64 block tiled over the volume; 4 dual steps
    (first launch, then the fused-final launch); the interior of each crop
    lies more than 5 voxels from crop faces that are not volume faces."""
    op, h = giga
    dev = torch.device("cuda:0")
    blk = synth.random_complex(synth.Stream(420), (32, 64, 64)).astype(np.complex64)
    v = torch.from_numpy(blk).to(dev).repeat(op.nz // 32, op.ny // 64, op.nx // 64)
    out = torch.empty_like(v)
    t_l1, t_tv, k = 0.3, 0.05, 4
    h.set_options(tv_dims=3)
    h.prox_fused_lasso(v, t_l1, t_tv, k, out)
    torch.cuda.synchronize()
    m = 8
    for (z0, y0, x0) in ((0, 0, 0), (500, 300, 700), (992, 984, 984)):
        z1, y1, x1 = min(op.nz, z0 + 32), min(op.ny, y0 + 40), min(op.nx, x0 + 40)
        crop = blk[np.ix_(np.arange(z0, z1) % 32, np.arange(y0, y1) % 64,
                          np.arange(x0, x1) % 64)].astype(np.complex128)
        ref = O.prox_fused_lasso(crop, t_l1, t_tv, k, 3)
        got = out[z0:z1, y0:y1, x0:x1].cpu().numpy()
        sl = tuple(slice(m if a > 0 else 0, (b - a) - (m if b < n else 0))
                   for a, b, n in ((z0, z1, op.nz), (y0, y1, op.ny), (x0, x1, op.nx)))
        assert rel_l2(got[sl], ref[sl]) <= OP_TOL, (z0, y0, x0)
    del v, out


def test_giga_first_iterate_on_a_crop(giga):
    """rihv_solve with one iteration from x_0 = 0 gives x_1 = prox(v),
    v = 2 tau H^H b, tau = 1/(2 nz). The oracle forms v on the crop's planes
    (one-plane adjoints of b) and its prox with the workload's 20 dual steps;
    the crop's interior lies more than 21 voxels from crop faces inside the
    volume, beyond the reach of 20 steps."""
    op, h = giga
    dev = torch.device("cuda:0")
    b = (0.5 + 0.1 * synth.random_complex(synth.Stream(430), (op.ny, op.nx)).real).astype(np.float32)
    h.set_options(tv_dims=3, n_inner=W.n_inner, check_every=0)
    x = torch.empty(op.shape, dtype=torch.complex64, device=dev)
    h.solve(b, W.lam_l1, W.lam_tv, 1, x)
    torch.cuda.synchronize()
    tau = 1.0 / (2 * op.nz)
    z0, y0, x0, n, m = 480, 400, 600, 64, 22
    v = np.stack([2 * tau * O.adjoint(b.astype(np.float64), slab(op, z0 + j))[0]
                  [y0:y0 + n, x0:x0 + n] for j in range(n)])
    ref = O.prox_fused_lasso(v, tau * W.lam_l1, tau * W.lam_tv, W.n_inner, 3)
    got = x[z0:z0 + n, y0:y0 + n, x0:x0 + n].cpu().numpy()
    inner = (slice(m, n - m),) * 3
    assert np.abs(ref[inner]).max() > 0
    assert rel_l2(got[inner], ref[inner]) <= 1e-4
    del x


def test_giga_sequence_stored_as_coo(giga):
    """Three frames of advected particles, 20 iterations each, every frame
    warm-started from the previous frame's COO form."""
    op, h = giga
    h.close()                                   # the sequence holds its own handle
    torch.cuda.empty_cache()
    res = coo_sequence.run(W, frames=3, iters=20, warm=True, log=lambda *_: None, keep=True)
    stored, x, hs = res["_stored"], res["_last"], res["_handle"]
    assert [r["warm"] for r in res["per_frame"]] == [False, True, True]
    assert res["stored_coo_bytes"] < res["stored_dense_bytes"], res["stored_coo_bytes"]
    assert all(r["nnz"] > 0 for r in res["per_frame"])
    # the last stored form is the last solution, exactly
    back = torch.empty_like(x)
    hs.coo_expand(*stored[-1], back)
    assert torch.equal(back, x)
    d_dense = hs.detect(x)
    d_coo = hs.detect_coo(*stored[-1])
    assert [(d["first"], d["nvox"]) for d in d_dense] == [(d["first"], d["nvox"]) for d in d_coo]
    assert len(d_coo) > 0
    print(json_line(res))
    hs.close()


def json_line(res):
    import json
    return json.dumps({k: v for k, v in res.items() if not k.startswith("_")})
