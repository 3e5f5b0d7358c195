"""Autograd wrappers: gradients through the hand-written kernels against the
FP64 oracle gradient and against central finite differences of the oracle's
objective."""
import numpy as np
import pytest
import torch

from oracle import rihv_oracle as O
from paper_1904_04884_gb300 import synth
from paper_1904_04884_gb300.autograd import hologram_adjoint, hologram_model
from paper_1904_04884_gb300.rihv import Rihv

pytestmark = pytest.mark.gpu

OP = O.Optics(nx=64, ny=48, nz=7, wavelength=632.8e-9, pitch=10e-6, z0=5e-3, dz=100e-6)


def _setup(seed):
    dev = torch.device("cuda:0")
    h = Rihv(OP.nx, OP.ny, OP.nz, OP.wavelength, OP.pitch, OP.z0, OP.dz)
    x = synth.random_complex(synth.Stream(seed), OP.shape)
    b = synth.Stream(seed + 1).normal(OP.nx * OP.ny).reshape(OP.ny, OP.nx)
    return dev, h, x, b


def test_data_term_gradient_matches_oracle():
    """grad of L = ||Hx - b||^2 via autograd equals the oracle's 2 H^H(Hx - b)."""
    dev, h, x, b = _setup(1)
    xt = torch.from_numpy(x.astype(np.complex64)).to(dev).requires_grad_(True)
    bt = torch.from_numpy(b.astype(np.complex64)).to(dev)
    loss = (hologram_model(xt, h) - bt).abs().pow(2).sum()
    loss.backward()
    # PyTorch's x.grad for real L is dL/dRe x + i dL/dIm x, here 2 H^H(Hx - b).
    g = xt.grad.cpu().numpy().astype(np.complex128)
    ref = O.grad_data(x.astype(np.complex64).astype(np.complex128), b, OP)
    assert np.linalg.norm(g - ref) / np.linalg.norm(ref) < 1e-5
    assert abs(loss.item() - O.data_term(x.astype(np.complex64).astype(np.complex128), b, OP)) \
        / loss.item() < 1e-5


def test_gradient_matches_finite_differences():
    """Re<grad, d> equals the FP64 central difference of the oracle objective."""
    dev, h, x, b = _setup(2)
    x = x.astype(np.complex64).astype(np.complex128)
    xt = torch.from_numpy(x.astype(np.complex64)).to(dev).requires_grad_(True)
    bt = torch.from_numpy(b.astype(np.complex64)).to(dev)
    (hologram_model(xt, h) - bt).abs().pow(2).sum().backward()
    g = xt.grad.cpu().numpy().astype(np.complex128)
    for s in (3, 4, 5):
        d = synth.random_complex(synth.Stream(100 + s), OP.shape)
        eps = 1e-5
        fd = (O.data_term(x + eps * d, b, OP) - O.data_term(x - eps * d, b, OP)) / (2 * eps)
        an = np.vdot(g, d).real
        assert abs(fd - an) / abs(fd) < 1e-5, (fd, an)


def test_adjoint_function_backward_is_forward():
    dev, h, x, b = _setup(3)
    r = synth.random_complex(synth.Stream(9), (OP.ny, OP.nx))
    rt = torch.from_numpy(r.astype(np.complex64)).to(dev).requires_grad_(True)
    c = synth.random_complex(synth.Stream(10), OP.shape)
    ct = torch.from_numpy(c.astype(np.complex64)).to(dev)
    # L = Re<c, H^H r> = Re<H c, r>; PyTorch's r.grad (dL/dRe r + i dL/dIm r)
    # is therefore H c.
    loss = (torch.conj(ct) * hologram_adjoint(rt, h)).real.sum()
    loss.backward()
    g = rt.grad.cpu().numpy().astype(np.complex128)
    ref = O.forward(c.astype(np.complex64).astype(np.complex128), OP)
    assert np.linalg.norm(g - ref) / np.linalg.norm(ref) < 1e-5


def test_autograd_runs_on_a_side_stream():
    dev, h, x, b = _setup(4)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        xt = torch.from_numpy(x.astype(np.complex64)).to(dev).requires_grad_(True)
        y = hologram_model(xt, h)
        y.abs().pow(2).sum().backward()
    torch.cuda.synchronize()
    assert torch.isfinite(xt.grad).all()
