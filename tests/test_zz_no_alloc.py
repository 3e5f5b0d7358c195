"""The allocation-free prox entry point against the regular one and the oracle.

rihv_prox_fused_lasso_noalloc serves callers that cannot allocate device
memory: hosts whose device memory is a fixed arena of their own, and services
that stop allocating after start-up so that no request can fail for lack of
memory. Its scratch is a static array inside the library. This test calls it
twice in a row through the C ABI, with different inputs and sizes so that
stale scratch contents from the first call would show, and compares each
result with rihv_prox_fused_lasso on a handle and with the FP64 oracle. It
also checks that the calls leave the device's free memory and torch's
allocation count unchanged. This file is collected last so that a failure
here does not hide the others.
"""
import numpy as np
import pytest
import torch

from oracle import rihv_oracle as O
from paper_1904_04884_gb300 import synth
from paper_1904_04884_gb300.rihv import Rihv, RihvError, rihv_prox_fused_lasso_noalloc

pytestmark = pytest.mark.gpu

OP_TOL = 1e-5


def _rel(a, b):
    a = np.asarray(a, np.complex128)
    b = np.asarray(b, np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _free_bytes():
    return torch.cuda.mem_get_info()[0]      # cudaMemGetInfo


@pytest.fixture(scope="module", autouse=True)
def first_call():
    """One call before the measured ones: the first call on a device looks up
    the scratch's address, which may load the library's module there (code
    and the static scratch itself), so device memory may change once."""
    dev = torch.device("cuda:0")
    v = torch.ones((2, 16, 16), dtype=torch.complex64, device=dev)
    rihv_prox_fused_lasso_noalloc(v, torch.empty_like(v), 2, 16, 16, 3, 0.1, 0.1, 2)
    torch.cuda.synchronize()


def _case(nx, ny, nz, seed, dims, k, t_l1, t_tv):
    dev = torch.device("cuda:0")
    v_np = synth.random_complex(synth.Stream(seed), (nz, ny, nx)).astype(np.complex64)
    v = torch.from_numpy(v_np).to(dev)
    h = Rihv(nx, ny, nz, 532e-9, 5e-6, 5e-3, 50e-6)
    h.set_options(tv_dims=dims)
    ref = torch.empty_like(v)
    h.prox_fused_lasso(v, t_l1, t_tv, k, ref)
    out = torch.full_like(v, float("nan"))
    torch.cuda.synchronize()
    alloc0, free0 = torch.cuda.memory_allocated(), _free_bytes()
    rihv_prox_fused_lasso_noalloc(v, out, nz, ny, nx, dims, t_l1, t_tv, k)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == alloc0
    assert _free_bytes() == free0
    oracle = O.prox_fused_lasso(v_np.astype(np.complex128), t_l1, t_tv, k, dims)
    return out.cpu().numpy(), ref.cpu().numpy(), oracle


def test_noalloc_matches_regular_prox_and_oracle_twice():
    assert torch.cuda.is_available()
    out1, ref1, or1 = _case(48, 24, 37, 11, 3, 20, 0.3, 0.05)
    assert np.isfinite(out1).all()
    assert _rel(out1, ref1) <= OP_TOL and _rel(out1, or1) <= OP_TOL
    out2, ref2, or2 = _case(64, 32, 9, 12, 2, 7, 0.2, 0.08)
    assert np.isfinite(out2).all()
    assert _rel(out2, ref2) <= OP_TOL and _rel(out2, or2) <= OP_TOL


def test_noalloc_rejects_oversized_volume_and_host_memory():
    dev = torch.device("cuda:0")
    v = torch.zeros((2, 1024, 1024), dtype=torch.complex64, device=dev)   # 2 Mi voxels
    with pytest.raises(RihvError) as e:
        rihv_prox_fused_lasso_noalloc(v, torch.empty_like(v), 2, 1024, 1024, 3, 0.1, 0.1, 2)
    assert e.value.status == 6 and "limit" in str(e.value)
    host = np.zeros((4, 16, 16), np.complex64)
    out = torch.empty((4, 16, 16), dtype=torch.complex64, device=dev)
    with pytest.raises(RihvError) as e:
        rihv_prox_fused_lasso_noalloc(host.ctypes.data, out, 4, 16, 16, 3, 0.1, 0.1, 2)
    assert e.value.status == 1


@pytest.mark.skipif(torch.cuda.device_count() < 2, reason="needs a second visible GPU")
def test_noalloc_rejects_memory_of_another_device():
    v = torch.zeros((4, 16, 16), dtype=torch.complex64, device="cuda:1")
    out = torch.empty((4, 16, 16), dtype=torch.complex64, device="cuda:0")
    with torch.cuda.device(0):
        with pytest.raises(RihvError) as e:
            rihv_prox_fused_lasso_noalloc(v, out, 4, 16, 16, 3, 0.1, 0.1, 2)
    assert e.value.status == 1
