"""The allocation-free prox entry point against the regular one.

rihv_prox_fused_lasso_noalloc serves callers that cannot allocate device
memory (for example code running during CUDA graph capture, or under another
framework's fixed memory arena): its scratch is a static array inside the
library. This test calls it twice in a row through the C ABI, with different
inputs and sizes so that stale scratch contents from the first call would
show, and compares each result with rihv_prox_fused_lasso on a handle.
This file is collected last so that a failure here does not hide the others.
"""
import numpy as np
import pytest
import torch

from paper_1904_04884_gb300 import synth
from paper_1904_04884_gb300.rihv import Rihv, RihvError, rihv_prox_fused_lasso_noalloc

pytestmark = pytest.mark.gpu

OP_TOL = 1e-5


def _rel(a, b):
    a = a.cpu().numpy().astype(np.complex128)
    b = b.cpu().numpy().astype(np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _case(nx, ny, nz, seed, dims, k, t_l1, t_tv):
    dev = torch.device("cuda:0")
    v = torch.from_numpy(synth.random_complex(synth.Stream(seed), (nz, ny, nx))
                         .astype(np.complex64)).to(dev)
    h = Rihv(nx, ny, nz, 532e-9, 5e-6, 5e-3, 50e-6)
    h.set_options(tv_dims=dims)
    ref = torch.empty_like(v)
    h.prox_fused_lasso(v, t_l1, t_tv, k, ref)
    out = torch.full_like(v, float("nan"))
    rihv_prox_fused_lasso_noalloc(v, out, nz, ny, nx, dims, t_l1, t_tv, k)
    torch.cuda.synchronize()
    return out, ref


def test_noalloc_matches_regular_prox_twice():
    assert torch.cuda.is_available()
    out1, ref1 = _case(48, 24, 37, 11, 3, 20, 0.3, 0.05)
    assert torch.isfinite(out1).all() and _rel(out1, ref1) <= OP_TOL
    out2, ref2 = _case(64, 32, 9, 12, 2, 7, 0.2, 0.08)
    assert torch.isfinite(out2).all() and _rel(out2, ref2) <= OP_TOL


def test_noalloc_rejects_oversized_volume():
    dev = torch.device("cuda:0")
    v = torch.zeros((2, 1024, 1024), dtype=torch.complex64, device=dev)   # 2 Mi voxels
    with pytest.raises(RihvError) as e:
        rihv_prox_fused_lasso_noalloc(v, torch.empty_like(v), 2, 1024, 1024, 3, 0.1, 0.1, 2)
    assert e.value.status == 6
