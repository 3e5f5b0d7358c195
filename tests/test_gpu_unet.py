"""The warm-start U-Net on the GPU against an FP64 composition of the oracle
layers (BF16 rounding applied at the same points as the GPU stores BF16), and
a short training run that must lower the loss."""
import numpy as np
import pytest
import torch

from oracle import unet_oracle as U
from paper_1904_04884_gb300 import nn
from paper_1904_04884_gb300.unet import LAYERS, WarmStartUNet

pytestmark = pytest.mark.gpu

DIMS = (4, 8, 16)


def r16(a):
    """Round to BF16 (as the GPU stores activations and gradients)."""
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).double().numpy()


def _oracle_forward_backward(net, x0, gout):
    W = {n: net.Wb[n].double().cpu().numpy() for n, *_ in LAYERS}
    b = {n: net.b[n].double().cpu().numpy() for n, *_ in LAYERS}
    d0 = DIMS
    d1 = tuple(v // 2 for v in d0)
    d2 = tuple(v // 4 for v in d0)
    x = x0.reshape(*d0, 16)
    conv = lambda n, t, relu=True: r16(U.relu(U.conv3d(t, W[n], b[n]))) if relu else U.conv3d(t, W[n], b[n])
    a = {}
    a["e1a"] = conv("e1a", x)
    a["s1"] = conv("e1b", a["e1a"])
    a["p1"] = r16(U.avgpool2(a["s1"]))
    a["e2a"] = conv("e2a", a["p1"])
    a["s2"] = conv("e2b", a["e2a"])
    a["p2"] = r16(U.avgpool2(a["s2"]))
    a["b1"] = conv("b1", a["p2"])
    a["b2"] = conv("b2", a["b1"])
    a["c2"] = np.concatenate([U.upsample2(a["b2"]), a["s2"]], axis=-1)
    a["d2a"] = conv("d2a", a["c2"])
    a["d2b"] = conv("d2b", a["d2a"])
    a["c1"] = np.concatenate([U.upsample2(a["d2b"]), a["s1"]], axis=-1)
    a["d1a"] = conv("d1a", a["c1"])
    a["d1b"] = conv("d1b", a["d1a"])
    out = conv("out", a["d1b"], relu=False)
    g = gout.reshape(*d0, 16)
    gw = {}

    def back(n, xin, g, y=None, dgrad=True):
        if y is not None:
            g = np.where(y > 0, g, 0.0)
        gw[n] = U.conv3d_wgrad(xin, g)
        return r16(U.conv3d_dgrad(g, W[n])) if dgrad else None

    g = back("out", a["d1b"], g)
    g = back("d1b", a["d1a"], g, a["d1b"])
    g = back("d1a", a["c1"], g, a["d1a"])
    gu1, gs1 = g[..., :32], g[..., 32:]
    g = r16(U.upsample2_grad(gu1))
    g = back("d2b", a["d2a"], g, a["d2b"])
    g = back("d2a", a["c2"], g, a["d2a"])
    gu2, gs2 = g[..., :64], g[..., 64:]
    g = r16(U.upsample2_grad(gu2))
    g = back("b2", a["b1"], g, a["b2"])
    g = back("b1", a["p2"], g, a["b1"])
    g = r16(r16(U.avgpool2_grad(g)) + gs2)
    g = back("e2b", a["e2a"], g, a["s2"])
    g = back("e2a", a["p1"], g, a["e2a"])
    g = r16(r16(U.avgpool2_grad(g)) + gs1)
    g = back("e1b", a["e1a"], g, a["s1"])
    back("e1a", x, g, a["e1a"], dgrad=False)
    return out, gw


def test_unet_forward_and_weight_gradients_match_oracle():
    dev = torch.device("cuda:0")
    net = WarmStartUNet(DIMS, seed=3)
    # give every layer non-trivial weights (the output layer starts small)
    for n, *_ in LAYERS:
        net._set(n, net.W[n] * 2.0 + 0.01, torch.linspace(-0.1, 0.1, net.b[n].numel()))
    g = torch.Generator().manual_seed(1)
    x0 = torch.randn(int(np.prod(DIMS)), 16, generator=g).to(torch.bfloat16)
    gout = (1e-2 * torch.randn(int(np.prod(DIMS)), 16, generator=g)).to(torch.bfloat16)
    out = net.forward(x0.to(dev))
    net.backward(gout.to(dev))
    torch.cuda.synchronize()
    assert net.errors() == 0
    ref_out, ref_gw = _oracle_forward_backward(net, x0.double().numpy(), gout.double().numpy())
    o = out.cpu().double().numpy()
    assert np.linalg.norm(o - ref_out.reshape(o.shape)) / np.linalg.norm(ref_out) < 2e-2
    for n, *_ in LAYERS:
        got = net.gW[n].cpu().double().numpy()
        ref = ref_gw[n]
        assert np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-30) < 5e-2, n


def test_training_lowers_the_loss():
    dev = torch.device("cuda:0")
    dims = (8, 16, 16)
    net = WarmStartUNet(dims, seed=5)
    g = torch.Generator().manual_seed(2)
    hb = torch.randn(*dims, dtype=torch.complex64, generator=g).to(dev)
    target = (0.5 * hb.real.abs()).to(torch.complex64).contiguous()
    losses = [net.train_step(hb, target, lr=3e-3).item() for _ in range(60)]
    torch.cuda.synchronize()
    assert net.errors() == 0
    assert losses[-1] < 0.5 * losses[0], (losses[0], losses[-1])
    x0 = torch.empty_like(hb)
    net.predict(hb, x0)
    assert torch.isfinite(x0).all()
