"""Degenerate inputs through the C ABI, against what the method fixes
exactly and against the FP64 oracle.

- A zero hologram: the minimiser is x = 0 and FISTA from 0 never leaves it
  (every gradient, prox and momentum term is 0), so the volume and the
  objective trace are exactly 0 and nothing is detected.
- No iterations: x_out is the start (x_0, or 0 without one), bit for bit.
- No regularisation (lambda_l1 = lambda_tv = 0): plain accelerated least
  squares, against the oracle's iterates; the data are fitted exactly, so
  both objective traces fall to their rounding floors.
- The prox of a zero volume is 0; of a constant volume c it is c shrunk by
  the soft threshold, c max(0, 1 - t_l1/|c|) (D c = 0, so every dual step
  stays at p = 0 and the TV prox returns c).
"""
import numpy as np
import pytest
import torch

from oracle import rihv_oracle as O
from paper_1904_04884_gb300 import synth, workloads
from paper_1904_04884_gb300.rihv import Rihv

pytestmark = pytest.mark.gpu

SOLVE_TOL = 1e-3
OP_TOL = 1e-5


def _dev():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch.device("cuda:0")


def _rel(a, b):
    a = np.asarray(a, np.complex128)
    b = np.asarray(b, np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _tiny():
    w = workloads.TINY
    op = O.Optics(*w.optics_tuple())
    return w, op, Rihv(op.nx, op.ny, op.nz, op.wavelength, op.pitch, op.z0, op.dz)


@pytest.mark.parametrize("dims", [3, 2])
def test_zero_hologram_keeps_zero(dims):
    w, op, h = _tiny()
    h.set_options(tv_dims=dims)
    b = np.zeros((op.ny, op.nx), np.float32)
    x = torch.full(op.shape, 1.0, dtype=torch.complex64, device=_dev())
    trace = np.full(3, -1.0)
    done = h.solve(b, w.lam_l1, w.lam_tv, 30, x, trace=trace)
    assert done == 30
    assert torch.count_nonzero(x).item() == 0
    assert np.array_equal(trace, np.zeros(3))
    assert h.detect(x, 2.0 / 256.0, 5) == []
    ref, tr = O.fista(b.astype(np.float64), op, w.lam_l1, w.lam_tv, 30, w.n_inner, dims=dims,
                      check_every=10)
    assert np.abs(ref).max() == 0.0 and [f for _, f in tr] == [0.0, 0.0, 0.0]
    h.close()


def test_zero_iterations_return_the_start():
    w, op, h = _tiny()
    b = synth.intensity_hologram(O.forward(w.opacity().astype(np.float64), op), w.sigma, w.noise())
    x0 = torch.from_numpy(synth.random_complex(synth.Stream(5), op.shape)
                          .astype(np.complex64)).to(_dev())
    x = torch.full_like(x0, 7.0)
    assert h.solve(b, w.lam_l1, w.lam_tv, 0, x, x0=x0) == 0
    assert torch.equal(x, x0)
    assert h.solve(b, w.lam_l1, w.lam_tv, 0, x) == 0
    assert torch.count_nonzero(x).item() == 0
    h.close()


def test_unregularised_solve_matches_oracle():
    w, op, h = _tiny()
    b = synth.intensity_hologram(O.forward(w.opacity().astype(np.float64), op), w.sigma, w.noise())
    x = torch.empty(op.shape, dtype=torch.complex64, device=_dev())
    trace = np.zeros(2)
    h.solve(b, 0.0, 0.0, 20, x, trace=trace)
    ref, tr = O.fista(b.astype(np.float64), op, 0.0, 0.0, 20, w.n_inner, check_every=10)
    assert _rel(x.cpu().numpy(), ref) <= SOLVE_TOL
    # With more unknowns than data (16 planes, one hologram) and no
    # regulariser the data are fitted exactly: F falls from ||b||^2 to the
    # rounding floor (about 1e-30 in FP64, 1e-11 in FP32 arithmetic), so the
    # traces agree to a tolerance relative to F(0) = ||b||^2, not to F.
    f0 = float(np.sum(b.astype(np.float64) ** 2))
    ref_tr = np.array([f for _, f in tr])
    assert np.abs(trace - ref_tr).max() <= 1e-9 * f0
    assert trace.max() <= 1e-9 * f0 and ref_tr.max() <= 1e-9 * f0
    h.close()


@pytest.mark.parametrize("dims", [3, 2])
def test_prox_of_zero_and_constant_volumes(dims):
    w, op, h = _tiny()
    h.set_options(tv_dims=dims)
    out = torch.full(op.shape, 3.0, dtype=torch.complex64, device=_dev())
    zero = torch.zeros(op.shape, dtype=torch.complex64, device=_dev())
    h.prox_fused_lasso(zero, 0.1, 0.3, 20, out)
    torch.cuda.synchronize()
    assert torch.count_nonzero(out).item() == 0
    c = 0.6 - 0.8j                          # |c| = 1
    const = torch.full(op.shape, c, dtype=torch.complex64, device=_dev())
    for k in (1, 2, 7, 20):
        h.prox_fused_lasso(const, 0.25, 0.3, k, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, np.full(op.shape, 0.75 * c), rtol=0, atol=1e-6)
        ref = O.prox_fused_lasso(np.full(op.shape, c, np.complex128), 0.25, 0.3, k, dims)
        assert _rel(got, ref) <= OP_TOL
    h.close()
