"""Full-solve parity at a size that runs the large-scale launch paths: a
512 x 512 x 40 slab of the 512x512x128 workload (its optics, discs and noise
on the first 40 planes), 10 FISTA iterations with 20 TV dual steps per prox,
the default schedule (two dual steps per launch, the last one with the fused
FISTA finalize), against the FP64 oracle's solve of the same hologram.

The fused-final launch reduces the restart product over its CTAs (compensated
FP32 per thread, FP64 across CTAs) and decides the restart on the device. At
this size it runs 423 CTAs over one z-chunk by default; the second case forces
8-plane z-chunks, so that every TV launch, the fused final one included,
spans 5 chunks (2,115 CTAs for the final launch). Both must give the oracle's
volume to 1e-3 (relative L2) and its objective trace to 1e-4.

The oracle's solve takes a few minutes on one host core; it runs once for
both cases.
"""
import numpy as np
import pytest
import torch

from oracle import rihv_oracle as O
from paper_1904_04884_gb300 import synth, workloads
from paper_1904_04884_gb300.rihv import Rihv

pytestmark = pytest.mark.gpu

PLANES = 40
ITERS = 10


def _rel(a, b):
    a = np.asarray(a, np.complex128)
    b = np.asarray(b, np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def slab():
    w = workloads.MID
    op = O.Optics(w.nx, w.ny, PLANES, w.wavelength, w.pitch, w.z0, w.dz)
    a = w.opacity()[:PLANES].astype(np.float64)
    b = synth.intensity_hologram(O.forward(a, op), w.sigma, w.noise())
    x_ref, tr_ref = O.fista(b.astype(np.float64), op, w.lam_l1, w.lam_tv, ITERS, w.n_inner,
                            check_every=1)
    return w, op, b, x_ref, np.array([f for _, f in tr_ref])


@pytest.mark.parametrize("zchunk", [0, 8])
def test_slab_solve_matches_oracle(slab, zchunk):
    w, op, b, x_ref, tr_ref = slab
    h = Rihv(op.nx, op.ny, op.nz, op.wavelength, op.pitch, op.z0, op.dz)
    h.set_options(n_inner=w.n_inner, check_every=1, tv_dims=w.tv_dims, tv_zchunk=zchunk)
    x = torch.empty(op.shape, dtype=torch.complex64, device="cuda:0")
    trace = np.zeros(ITERS)
    done = h.solve(b, w.lam_l1, w.lam_tv, ITERS, x, trace=trace)
    assert done == ITERS
    xs = x.cpu().numpy()
    err = _rel(xs, x_ref)
    print(f"zchunk {zchunk}: volume rel L2 {err:.3g}, trace max rel "
          f"{np.max(np.abs(trace - tr_ref) / np.abs(tr_ref)):.3g}")
    assert err <= 1e-3
    np.testing.assert_allclose(trace, tr_ref, rtol=1e-4)
