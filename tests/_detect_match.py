"""Comparison of two particle-detection lists by the detection parity rule.

Two volumes xa, xb and their detections da, db (lists of dicts with
``centroid`` (x, y, z), ``nvox`` and ``first``, as the oracle and the GPU
binding return them). Components are matched one to one by centroid, within
0.5 voxel, nearest first. A component may be unmatched, or matched with a
different voxel count, only if it is exempt: one of its voxels, or one of
their 26 neighbours, has |x| within ``band`` of the detection threshold in
either volume (a voxel near the threshold may fall on either side of it,
which changes the components it belongs to or touches; every other voxel is
decided alike in both volumes). Nothing here calls the oracle or the library.
"""
from __future__ import annotations

import numpy as np
from scipy import ndimage
from scipy.spatial import cKDTree

STRUCT = np.ones((3, 3, 3), dtype=bool)


def _mask_f32(x, rel):
    xr = np.ascontiguousarray(np.real(x), dtype=np.float32)
    xi = np.ascontiguousarray(np.imag(x), dtype=np.float32)
    m2 = xr * xr + xi * xi
    thr2 = np.float32(np.float32(rel) * np.float32(rel)) * np.float32(m2.max())
    return m2 > thr2


def edge_mask(x, rel, band):
    """Voxels whose |x| lies within `band` of rel * max|x| (FP64)."""
    m = np.abs(np.asarray(x, np.complex128))
    return np.abs(m - rel * m.max()) < band


def compare(xa, da, xb, db, rel, band):
    """Returns a dict: matched, exempt (components excused by the band), bad
    (components that differ without touching it), and the counts."""
    near = ndimage.binary_dilation(edge_mask(xa, rel, band) | edge_mask(xb, rel, band),
                                   structure=STRUCT)
    labels = []
    for x in (xa, xb):
        lab, _ = ndimage.label(_mask_f32(x, rel), structure=STRUCT)
        labels.append(lab)
    touched = []
    for lab in labels:
        hit = np.unique(lab[near & (lab > 0)])
        touched.append(set(int(v) for v in hit))

    def is_exempt(side, d):
        lab = labels[side]
        first = np.unravel_index(int(d["first"]), lab.shape)
        return int(lab[first]) in touched[side]

    ca = np.array([d["centroid"] for d in da], dtype=np.float64).reshape(-1, 3)
    cb = np.array([d["centroid"] for d in db], dtype=np.float64).reshape(-1, 3)
    pairs = []
    if len(ca) and len(cb):
        tree = cKDTree(cb)
        dist, idx = tree.query(ca, k=1, distance_upper_bound=0.5)
        order = np.argsort(dist)
        used_b = set()
        for i in order:
            j = int(idx[i])
            if np.isfinite(dist[i]) and j not in used_b:
                used_b.add(j)
                pairs.append((int(i), j))
    ma = {i for i, _ in pairs}
    mb = {j for _, j in pairs}
    exempt, bad = [], []
    for i, j in pairs:
        if da[i]["nvox"] != db[j]["nvox"]:
            (exempt if is_exempt(0, da[i]) or is_exempt(1, db[j]) else bad).append(("nvox", i, j))
    for i, d in enumerate(da):
        if i not in ma:
            (exempt if is_exempt(0, d) else bad).append(("a", i))
    for j, d in enumerate(db):
        if j not in mb:
            (exempt if is_exempt(1, d) else bad).append(("b", j))
    return {"matched": len(pairs), "n_a": len(da), "n_b": len(db), "exempt": len(exempt),
            "bad": bad, "band": band}
