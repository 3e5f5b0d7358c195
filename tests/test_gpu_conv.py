"""tcgen05 convolution kernels of the warm-start network against the FP64
oracle, on BF16-rounded inputs (so only the accumulation order differs)."""
import numpy as np
import pytest
import torch

from oracle import unet_oracle as U
from paper_1904_04884_gb300 import nn

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")
TOL = 1e-5         # FP32 accumulation of BF16 products vs FP64


def _bf16(shape, seed, scale=1.0):
    g = torch.Generator().manual_seed(seed)
    return (scale * torch.randn(*shape, generator=g)).to(torch.bfloat16)


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = [((5, 6, 40), 16, 16), ((4, 8, 16), 32, 64), ((3, 4, 32), 96, 32), ((2, 3, 7), 48, 16),
         ((6, 6, 6), 16, 32), ((2, 5, 200), 32, 16), ((3, 9, 130), 16, 64)]


@pytest.mark.parametrize("dims,cin,cout", CASES)
def test_conv_forward_matches_oracle(dims, cin, cout):
    nvox = int(np.prod(dims))
    x = _bf16((nvox, cin), 1)
    w = _bf16((cout, 27, cin), 2, 0.1)
    b = torch.randn(cout, generator=torch.Generator().manual_seed(3))
    err = torch.zeros(1, dtype=torch.int32, device=DEV)
    y = torch.empty((nvox, cout), dtype=torch.float32, device=DEV)
    nn.conv3d(x.to(DEV), w.to(DEV), b.to(DEV), y, dims, cin, cout, relu=False, err=err)
    torch.cuda.synchronize()
    assert err.item() == 0
    ref = U.conv3d(x.float().numpy().reshape(*dims, cin), w.float().numpy(), b.numpy())
    assert _rel(y.cpu().numpy(), ref.reshape(nvox, cout)) <= TOL
    # BF16 output with ReLU: within BF16 rounding of the FP64 result
    yb = torch.empty((nvox, cout), dtype=torch.bfloat16, device=DEV)
    nn.conv3d(x.to(DEV), w.to(DEV), b.to(DEV), yb, dims, cin, cout, relu=True, err=err)
    r = np.maximum(ref.reshape(nvox, cout), 0)
    got = yb.float().cpu().numpy()
    assert np.all(np.abs(got - r) <= 2.0 ** -8 * np.abs(r) + 1e-6)


@pytest.mark.parametrize("dims,cin,cout", CASES)
def test_conv_dgrad_matches_oracle(dims, cin, cout):
    nvox = int(np.prod(dims))
    gy = _bf16((nvox, cout), 4)
    w = _bf16((cout, 27, cin), 5, 0.1)
    err = torch.zeros(1, dtype=torch.int32, device=DEV)
    gx = torch.empty((nvox, cin), dtype=torch.float32, device=DEV)
    nn.conv3d_dgrad(gy.to(DEV), w.to(DEV), gx, dims, cin, cout, err)
    torch.cuda.synchronize()
    assert err.item() == 0
    ref = U.conv3d_dgrad(gy.float().numpy().reshape(*dims, cout), w.float().numpy())
    assert _rel(gx.cpu().numpy(), ref.reshape(nvox, cin)) <= TOL


@pytest.mark.parametrize("dims,cin,cout", CASES)
def test_conv_wgrad_matches_oracle(dims, cin, cout):
    if cout > 64:
        pytest.skip("weight gradient supports c_out <= 64")
    nvox = int(np.prod(dims))
    x = _bf16((nvox, cin), 6)
    gy = _bf16((nvox, cout), 7)
    err = torch.zeros(1, dtype=torch.int32, device=DEV)
    gw = torch.empty((cout, 27, cin), dtype=torch.float32, device=DEV)
    work = torch.empty(nn.wgrad_workspace_bytes(dims, cin, cout) // 4 + 4, dtype=torch.float32,
                       device=DEV)
    nn.conv3d_wgrad(x.to(DEV), gy.to(DEV), gw, dims, cin, cout, work, err)
    torch.cuda.synchronize()
    assert err.item() == 0
    ref = U.conv3d_wgrad(x.float().numpy().reshape(*dims, cin), gy.float().numpy().reshape(*dims, cout))
    assert _rel(gw.cpu().numpy(), ref) <= TOL


def test_pool_upsample_concat_relu_and_bias_grad():
    dims = (4, 6, 8)
    c = 16
    nvox = int(np.prod(dims))
    x = _bf16((nvox, c), 8)
    xd = x.to(DEV)
    pooled = torch.empty((nvox // 8, c), dtype=torch.bfloat16, device=DEV)
    nn.avgpool2(xd, pooled, dims, c)
    ref = U.avgpool2(x.float().numpy().reshape(*dims, c))
    np.testing.assert_allclose(pooled.float().cpu().numpy().reshape(ref.shape), ref, rtol=8e-3, atol=1e-3)
    up = torch.empty((nvox, c), dtype=torch.bfloat16, device=DEV)
    nn.upsample2(pooled, up, (2, 3, 4), c)
    np.testing.assert_array_equal(up.float().cpu().numpy().reshape(*dims, c),
                                  U.upsample2(pooled.float().cpu().numpy().reshape(2, 3, 4, c)))
    g = torch.empty((nvox // 8, c), dtype=torch.bfloat16, device=DEV)
    nn.upsample2_grad(up, g, (2, 3, 4), c)
    ref = U.upsample2_grad(up.float().cpu().numpy().reshape(*dims, c))
    np.testing.assert_allclose(g.float().cpu().numpy().reshape(ref.shape), ref, rtol=8e-3, atol=1e-3)
    cat = torch.empty((nvox, 2 * c), dtype=torch.bfloat16, device=DEV)
    nn.concat(xd, up, cat, nvox, c, c)
    a2 = torch.empty_like(xd)
    b2 = torch.empty_like(up)
    nn.split(cat, a2, b2, nvox, c, c)
    assert torch.equal(a2, xd) and torch.equal(b2, up)
    rg = torch.empty_like(xd)
    nn.relu_grad(up, xd, rg)
    assert torch.equal(rg, torch.where(xd.float() > 0, up, torch.zeros_like(up)))
    gb = torch.empty(c, dtype=torch.float32, device=DEV)
    work = torch.empty(256 * c, dtype=torch.float64, device=DEV)
    nn.bias_grad(xd, gb, nvox, c, work)
    np.testing.assert_allclose(gb.cpu().numpy(), x.double().numpy().sum(axis=0), rtol=1e-6, atol=1e-5)


@pytest.mark.parametrize("c", [16, 32, 64, 48])
def test_bias_grad_large(c):
    """gb[c] = sum over voxels of gy[v][c] on a ragged voxel count (the
    vectorised reduction over 8-channel words), against an FP64 sum."""
    nvox = 300_007
    gy = _bf16((nvox, c), 9 + c)
    gb = torch.empty(c, dtype=torch.float32, device=DEV)
    work = torch.empty(256 * c, dtype=torch.float64, device=DEV)
    nn.bias_grad(gy.to(DEV), gb, nvox, c, work)
    torch.cuda.synchronize()
    ref = gy.double().numpy().sum(axis=0)
    np.testing.assert_allclose(gb.cpu().numpy(), ref, rtol=1e-6, atol=1e-4)
