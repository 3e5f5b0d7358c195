"""Failure detection on the GPU without a fault: the bounded mbarrier wait
that guards every TMA tile arrival in the TV kernels is made to run out on a
barrier that nothing arrives on; the library must report RIHV_ERR_TIMEOUT and
leave the CUDA context usable (a forward call afterwards still matches the
oracle)."""
import numpy as np
import pytest
import torch

from oracle import rihv_oracle as O
from paper_1904_04884_gb300 import synth
from paper_1904_04884_gb300.rihv import Rihv

pytestmark = pytest.mark.gpu

TIMEOUT, INVALID = 5, 1


def test_bounded_wait_gives_up_and_the_context_survives():
    op = O.Optics(nx=64, ny=64, nz=4, wavelength=632.8e-9, pitch=10e-6, z0=5e-3, dz=100e-6)
    h = Rihv(op.nx, op.ny, op.nz, op.wavelength, op.pitch, op.z0, op.dz)
    for polls in (1, 4096, 1 << 16):
        assert h.rihv_selftest_bounded_wait(polls) == TIMEOUT
        assert b"gave up" in h.L.rihv_last_error(h.h)
    assert h.rihv_selftest_bounded_wait(0) == INVALID
    assert h.rihv_selftest_bounded_wait((1 << 22) + 1) == INVALID
    # the context still works, and the error flag was cleared for the next call
    x = synth.random_complex(synth.Stream(5), op.shape)
    out = torch.empty((op.ny, op.nx), dtype=torch.complex64, device="cuda:0")
    h.forward(torch.from_numpy(x.astype(np.complex64)).to("cuda:0"), out)
    torch.cuda.synchronize()
    ref = O.forward(x, op)
    assert np.linalg.norm(out.cpu().numpy() - ref) / np.linalg.norm(ref) <= 1e-5
    vol = torch.empty(op.shape, dtype=torch.complex64, device="cuda:0")
    h.prox_fused_lasso(torch.from_numpy(x.astype(np.complex64)).to("cuda:0"), 0.1, 0.05, 4, vol)
    torch.cuda.synchronize()
    assert np.isfinite(vol.cpu().numpy()).all()
