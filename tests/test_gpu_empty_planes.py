"""Empty-plane skipping in the forward propagation (Section 2: the volume is
sparse and each plane propagates on its own, so an all-zero plane of y_k or
x_k adds nothing to the z-sum and its FFTs can be left out).

The skip is exact, so solves with it on and off must agree to the bit, alone,
from a warm start and inside a batched graph; the problem is chosen so that
the solution has planes that are exactly zero (strong weights; the oracle's
30-iteration solution leaves 5 of its 16 planes empty), and the result must
also match the oracle."""
import numpy as np
import pytest
import torch

from oracle import rihv_oracle as O
from paper_1904_04884_gb300 import synth
from paper_1904_04884_gb300.rihv import Batch, Rihv

pytestmark = pytest.mark.gpu

LAM_L1, LAM_TV = 2.0, 0.5
ITERS = 30


def _problem(nz=16):
    op = O.Optics(nx=64, ny=64, nz=nz, wavelength=632.8e-9, pitch=10e-6, z0=5e-3, dz=100e-6)
    a = np.zeros(op.shape)
    a[4, 20:23, 30:33] = 1.0
    a[11, 40:44, 10:13] = 1.0
    b = synth.intensity_hologram(O.forward(a, op), 0.01, synth.Stream(3).normal(op.nx * op.ny))
    return op, b.astype(np.float32)


def _handle(op, **opts):
    h = Rihv(op.nx, op.ny, op.nz, op.wavelength, op.pitch, op.z0, op.dz)
    h.set_options(check_every=5, **opts)
    return h


def _solve(op, b, skip, dims=3, x0=None):
    h = _handle(op, tv_dims=dims, skip_empty_planes=skip)
    x = torch.empty(op.shape, dtype=torch.complex64, device="cuda:0")
    tr = np.zeros(ITERS // 5)
    n = h.solve(b, LAM_L1, LAM_TV, ITERS, x, x0=x0, trace=tr)
    torch.cuda.synchronize()
    return h, x, tr, n


def _empty_planes(h, x):
    off = h.coo_compact(x)[0].cpu().numpy()
    return int(np.count_nonzero(np.diff(off) == 0))


@pytest.mark.parametrize("dims", [3, 2])
def test_skip_is_exact(dims):
    op, b = _problem()
    h, x_on, tr_on, n_on = _solve(op, b, 1, dims)
    _, x_off, tr_off, n_off = _solve(op, b, 0, dims)
    assert _empty_planes(h, x_on) >= 1          # the skip was exercised
    assert torch.equal(x_on, x_off)
    assert np.array_equal(tr_on, tr_off) and n_on == n_off


def test_skip_from_a_warm_start():
    op, b = _problem()
    x0 = np.zeros(op.shape, np.complex64)
    x0[4, 18:25, 28:35] = 0.5                   # two planes occupied, the rest zero
    x0[12, 5:9, 5:9] = 0.25j
    x0d = torch.from_numpy(x0).to("cuda:0")
    _, x_on, tr_on, _ = _solve(op, b, 1, x0=x0d)
    _, x_off, tr_off, _ = _solve(op, b, 0, x0=x0d)
    assert torch.equal(x_on, x_off)
    assert np.array_equal(tr_on, tr_off)


def test_skip_matches_the_oracle():
    op, b = _problem()
    h, x, tr, _ = _solve(op, b, 1)
    ref, ref_tr = O.fista(b.astype(np.float64), op, LAM_L1, LAM_TV, ITERS, 20, check_every=5)
    got = x.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-3
    assert np.allclose(tr, [f for _, f in ref_tr], rtol=1e-4)
    # the oracle's solution has all-zero planes too
    assert np.count_nonzero(np.abs(ref).sum(axis=(1, 2)) == 0) >= 1


def test_skip_inside_a_batched_graph():
    op, b = _problem()
    hs = [_handle(op, skip_empty_planes=1), _handle(op, skip_empty_planes=0)]
    outs = [torch.empty(op.shape, dtype=torch.complex64, device="cuda:0") for _ in hs]
    trs = [np.zeros(ITERS // 5) for _ in hs]
    batch = Batch(hs)
    for _ in range(2):                          # the second launch reuses the graph
        batch.solve([b, b], LAM_L1, LAM_TV, ITERS, outs, traces=trs)
        torch.cuda.synchronize()
        assert torch.equal(outs[0], outs[1])
        assert np.array_equal(trs[0], trs[1])
    _, x_ref, tr_ref, _ = _solve(op, b, 0)
    assert torch.equal(outs[0], x_ref)
    assert np.array_equal(trs[0], tr_ref)
