"""Detection on the per-plane COO form (rihv_detect_coo) against detection on
the dense volume (rihv_detect) and the oracle's detection: the same
components in the same order with the same sizes, centroids to FP64
summation order. Covers ragged planes, empty planes and volumes, components
that cross plane and row boundaries, and the tiny workload's solution."""
import numpy as np
import pytest
import torch

from oracle import rihv_oracle as O
from paper_1904_04884_gb300 import synth, workloads
from paper_1904_04884_gb300.rihv import Rihv, RihvError

pytestmark = pytest.mark.gpu

REL = 2.0 / 256.0


def handle(shape):
    nz, ny, nx = shape
    return Rihv(nx, ny, nz, 532e-9, 5e-6, 5e-3, 50e-6)


def blobby(shape, seed, density=0.02):
    """Sparse volume: random blobs (3x3x3 smoothing of a sparse seed field)
    plus isolated weak noise, complex."""
    st = synth.Stream(seed)
    n = int(np.prod(shape))
    seedf = (st.uniform(n).reshape(shape) < density).astype(np.float64)
    from scipy import ndimage
    blobs = ndimage.uniform_filter(seedf, size=3, mode="constant")
    noise = 0.01 * (st.uniform(n).reshape(shape) < 0.05)
    ph = np.exp(2j * np.pi * st.uniform(n).reshape(shape))
    return ((blobs + noise) * ph).astype(np.complex64)


def same(d1, d2):
    assert [(d["first"], d["nvox"]) for d in d1] == [(d["first"], d["nvox"]) for d in d2]
    if d1:
        np.testing.assert_allclose([d["centroid"] for d in d1], [d["centroid"] for d in d2],
                                   atol=1e-6)


@pytest.mark.parametrize("shape,seed", [((9, 48, 48), 1), ((16, 64, 64), 2), ((3, 24, 16), 3),
                                        ((1, 32, 32), 4)])
@pytest.mark.parametrize("min_vox", [0, 5])
def test_coo_detection_matches_dense_and_oracle(shape, seed, min_vox):
    x = blobby(shape, seed)
    if shape[0] > 2:
        x[shape[0] // 2] = 0                              # an empty plane
    h = handle(shape)
    xd = torch.from_numpy(x).cuda()
    off, rows, cols, vals = h.coo_compact(xd)
    d_coo = h.detect_coo(off, rows, cols, vals, REL, min_vox)
    d_dense = h.detect(xd, REL, min_vox)
    d_ref = O.detect(x, REL, min_vox)
    assert len(d_ref) > 0
    same(d_coo, d_dense)
    same(d_coo, d_ref)


def test_coo_detection_of_a_solution():
    w = workloads.TINY
    op = O.Optics(*w.optics_tuple())
    b = synth.intensity_hologram(O.forward(w.opacity().astype(np.float64), op), w.sigma,
                                 w.noise())
    h = Rihv(*w.optics_tuple())
    x = torch.empty(op.shape, dtype=torch.complex64, device="cuda")
    h.solve(b, w.lam_l1, w.lam_tv, w.iters, x)
    off, rows, cols, vals = h.coo_compact(x)
    d_coo = h.detect_coo(off, rows, cols, vals)
    same(d_coo, h.detect(x))
    same(d_coo, O.detect(x.cpu().numpy(), REL, 5))
    assert len(d_coo) > 0


def test_coo_detection_empty_and_invalid():
    shape = (4, 16, 32)
    h = handle(shape)
    off, rows, cols, vals = h.coo_compact(torch.zeros(shape, dtype=torch.complex64, device="cuda"))
    assert h.detect_coo(off, rows, cols, vals) == []
    x = torch.from_numpy(blobby(shape, 9, 0.05)).cuda()
    off, rows, cols, vals = h.coo_compact(x)
    bad = off.clone()
    bad[-1] += 1                                           # last offset != nnz
    with pytest.raises(RihvError) as e:
        h.detect_coo(bad, rows, cols, vals)
    assert e.value.status == 1
