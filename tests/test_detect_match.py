"""The detection comparison used by the parity tests, on hand-made volumes:
it accepts identical detections, excuses a component only when it touches a
voxel near the threshold, and flags any other difference."""
import numpy as np

from oracle import rihv_oracle as O
from tests import _detect_match as M

REL = 2.0 / 256.0


def _blobs():
    x = np.zeros((8, 24, 24), np.complex128)
    x[2:4, 3:6, 3:6] = 1.0                 # 18 voxels
    x[5:7, 12:15, 14:17] = 0.8 + 0.3j      # 18 voxels
    x[1:3, 18:21, 4:7] = 0.5               # 18 voxels
    return x


def test_identical_volumes_match_without_exemptions():
    x = _blobs()
    d = O.detect(x, REL, 5)
    r = M.compare(x, d, x.copy(), O.detect(x.copy(), REL, 5), REL, 1e-3)
    assert r["matched"] == len(d) == 3 and r["exempt"] == 0 and r["bad"] == []


def test_voxel_near_threshold_is_excused():
    """A voxel at the threshold in one volume and just above it in the other
    joins a blob on one side only: the blob's size differs, and it is
    excused because it touches that voxel."""
    x = _blobs()
    y = x.copy()
    thr = REL * 1.0
    x[2, 6, 5] = thr * (1 - 1e-4)      # below: not part of the blob
    y[2, 6, 5] = thr * (1 + 1e-4)      # above: part of it
    r = M.compare(x, O.detect(x, REL, 5), y, O.detect(y, REL, 5), REL, 1e-3)
    assert r["bad"] == [] and r["exempt"] == 1


def test_moved_or_missing_component_is_flagged():
    x = _blobs()
    y = x.copy()
    y[1:3, 18:21, 4:7] = 0.0
    y[1:3, 18:21, 8:11] = 0.5           # the third blob moved by 4 voxels
    r = M.compare(x, O.detect(x, REL, 5), y, O.detect(y, REL, 5), REL, 1e-3)
    assert len(r["bad"]) == 2 and r["matched"] == 2
    z = x.copy()
    z[5:7, 12:15, 14:17] = 0.0          # one blob gone
    r = M.compare(x, O.detect(x, REL, 5), z, O.detect(z, REL, 5), REL, 1e-3)
    assert len(r["bad"]) == 1
