"""What the trained warm start gains: on held-out seeds (training used seeds
1-256), FISTA started from the network's prediction reaches the objective
tolerance F* (1 + 1e-3) in fewer iterations than FISTA from zero, where F* is
the objective of a 600-iteration plain solve. The same holds when the warm
starts are solved together as one batched CUDA graph."""
import numpy as np
import pytest
import torch

from paper_1904_04884_gb300 import warmstart as W
from paper_1904_04884_gb300.rihv import Batch
from paper_1904_04884_gb300.unet import WarmStartUNet

pytestmark = pytest.mark.gpu

SEEDS = (20001, 20003)


@pytest.fixture(scope="module")
def cases():
    dev = torch.device("cuda:0")
    net = WarmStartUNet.load(W.DEFAULT_WEIGHTS)
    h = W.handle(W.SPEC)
    out = []
    for s in SEEDS:
        b, hb = W.make_sample(h, W.SPEC, s, dev)
        f_star = W.reference_objective(h, b, W.SPEC)
        x0 = torch.empty(W.SPEC.shape, dtype=torch.complex64, device=dev)
        net.predict(hb, x0)
        it_plain, _, xp = W.iterations_to_tolerance(h, b, W.SPEC, None, f_star)
        it_warm, _, xw = W.iterations_to_tolerance(h, b, W.SPEC, x0, f_star)
        out.append(dict(seed=s, b=b, x0=x0, f_star=f_star, it_plain=it_plain, it_warm=it_warm,
                        det_plain=len(h.detect(xp)), det_warm=len(h.detect(xw))))
    assert net.errors() == 0
    return out


def test_warm_start_needs_fewer_iterations(cases):
    for c in cases:
        assert c["it_warm"] < c["it_plain"], c
    assert sum(c["it_warm"] for c in cases) <= 0.85 * sum(c["it_plain"] for c in cases)


def test_warm_and_plain_detections_agree(cases):
    for c in cases:
        assert abs(c["det_warm"] - c["det_plain"]) <= 0.1 * max(c["det_plain"], 10), c


def test_batched_warm_starts_reach_the_tolerance(cases):
    """The warm starts solved together as one batched graph, each hologram
    with its own stop test inside the graph, stop after the same number of
    iterations as the individual warm solves, at the tolerance."""
    dev = torch.device("cuda:0")
    hs = [W.handle(W.SPEC, check_every=10, f_star=c["f_star"], tol=1e-3) for c in cases]
    outs = [torch.empty(W.SPEC.shape, dtype=torch.complex64, device=dev) for _ in cases]
    traces = [np.zeros(60) for _ in cases]
    batch = Batch(hs)
    batch.solve([c["b"] for c in cases], W.SPEC.lam_l1, W.SPEC.lam_tv, 600, outs,
                x0s=[c["x0"] for c in cases], traces=traces)
    its = batch.iterations()
    for c, tr, it in zip(cases, traces, its):
        assert it == c["it_warm"], (c["seed"], it, c["it_warm"])
        assert tr[it // 10 - 1] <= c["f_star"] * (1 + 1e-3) + 1e-9, (c["seed"], tr[it // 10 - 1])
    batch.close()
