"""Pins of the oracle's detection: labelling against a brute-force flood fill,
centroids of symmetric blobs, the minimum-volume filter and the strict
threshold."""
import numpy as np

from oracle import rihv_oracle as O
from tests import _brute as B


def test_labelling_matches_flood_fill():
    rng = np.random.default_rng(0)
    for trial, shape in enumerate([(6, 7, 8), (16, 16, 16), (3, 16, 11), (1, 9, 9)]):
        x = rng.random(shape) * (rng.random(shape) < 0.12)
        x = x + 1e-12            # nothing exactly zero; threshold does the masking
        comps = B.flood_fill_components(O.detection_mask(x, 0.05))
        det = O.detect(x, 0.05, min_vox=0)
        assert len(det) == len(comps)
        for d, c in zip(det, comps):
            assert d["first"] == c[0]
            assert d["nvox"] == len(c)
            kz, jy, ix = np.unravel_index(c, shape)
            w = np.abs(x.ravel()[c])
            np.testing.assert_allclose(d["centroid"],
                                       ((w * ix).sum() / w.sum(), (w * jy).sum() / w.sum(),
                                        (w * kz).sum() / w.sum()), rtol=1e-12)


def test_symmetric_blob_centroid_is_centre():
    x = np.zeros((9, 11, 13), complex)
    k, j, i = 4, 5, 6
    for dk in (-1, 0, 1):
        for dj in (-1, 0, 1):
            for di in (-1, 0, 1):
                x[k + dk, j + dj, i + di] = 1.0 / (1 + abs(dk) + abs(dj) + abs(di))
    d = O.detect(x, 0.01, 5)
    assert len(d) == 1
    np.testing.assert_allclose(d[0]["centroid"], (6.0, 5.0, 4.0), atol=1e-13)
    assert d[0]["nvox"] == 27


def test_min_volume_filter_and_diagonal_connectivity():
    x = np.zeros((8, 8, 8))
    # 5 voxels along a 3D diagonal: one 26-connected component, dropped (<= 5)
    for t in range(5):
        x[t, t, t] = 1.0
    # 6 voxels in a row: kept
    x[7, 0, :6] = 1.0
    d = O.detect(x, 0.5, 5)
    assert len(d) == 1 and d[0]["nvox"] == 6
    d0 = O.detect(x, 0.5, 0)
    assert sorted(c["nvox"] for c in d0) == [5, 6]


def test_threshold_is_strict_and_float32():
    # max |x| = 2; rel = 1/4 -> threshold 0.5 exactly; a voxel at 0.5 is out.
    x = np.zeros((1, 4, 4))
    x[0, 0, 0] = 2.0
    x[0, 3, 3] = 0.5
    x[0, 3, 2] = 0.5000001
    m = O.detection_mask(x, 0.25)
    assert m[0, 0, 0] and not m[0, 3, 3] and m[0, 3, 2]


def test_threshold_decision_rounds_each_operation_to_float32():
    """A voxel whose float32 and float64 decisions differ. max|x| = 1 and
    rel = 2^-7 give the threshold square 2^-14 exactly in either precision.
    The voxel 2^-7 + 2^-20 i has |x|^2 = 2^-14 + 2^-40: above the threshold
    in float64, but in float32 the sum re*re + im*im rounds to 2^-14 (2^-40
    is below half an ulp of 2^-14, which is 2^-38), not above it. The
    decision is the float32 one (strict >, each operation rounded)."""
    x = np.zeros((1, 2, 2), complex)
    x[0, 0, 0] = 1.0
    x[0, 1, 1] = 2.0 ** -7 + 1j * 2.0 ** -20
    x[0, 1, 0] = 2.0 ** -7 + 1j * 2.0 ** -18      # 2^-36 survives the float32 sum
    assert abs(x[0, 1, 1]) ** 2 > 2.0 ** -14
    m = O.detection_mask(x, 2.0 ** -7)
    assert m[0, 0, 0] and not m[0, 1, 1] and m[0, 1, 0]


def test_empty_detection():
    assert O.detect(np.zeros((2, 3, 4)), 0.1, 5) == []
