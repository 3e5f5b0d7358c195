"""Host logic of the workload runner's detection scoring (no GPU)."""
import numpy as np

from paper_1904_04884_gb300 import workloads
from paper_1904_04884_gb300.run_workload import match


def _as_detections(d, dx=0.0, dz=0.0):
    return [dict(centroid=(x - 0.5 + dx, y - 0.5, z + dz)) for x, y, z in zip(d.x, d.y, d.z)]


def test_exact_centres_match_every_disc():
    d = workloads.ALL["fista_mid_512x512x128"].discs()
    assert match(_as_detections(d), d, 2.0, 5.0) == (1.0, 1.0)


def test_window_edges():
    d = workloads.ALL["fista_mid_512x512x128"].discs()
    r, p = match(_as_detections(d, dx=1.9, dz=4.9), d, 2.0, 5.0)
    assert r == 1.0 and p == 1.0
    # outside the window on either axis: matches only by chance coincidence
    r, p = match(_as_detections(d, dx=30.0), d, 2.0, 5.0)
    assert r < 0.05 and p < 0.05
    r, p = match(_as_detections(d, dz=40.0), d, 2.0, 5.0)
    assert r < 0.05 and p < 0.05


def test_false_detections_lower_precision_only():
    d = workloads.ALL["fista_mid_512x512x128"].discs()
    far = [dict(centroid=(-100.0 - k, -100.0, 0.0)) for k in range(len(d))]
    r, p = match(_as_detections(d) + far, d, 2.0, 5.0)
    assert r == 1.0 and abs(p - 0.5) < 1e-12
    assert match([], d, 2.0, 5.0) == (0.0, 0.0)


def test_discs_are_the_rasterised_draws():
    w = workloads.ALL["fista_tiny_64x64x16"]
    d = w.discs()
    vol = w.opacity()
    for x, y, z in zip(d.x, d.y, d.z):
        assert vol[int(z), int(y), int(x)] > 0.0
    assert np.count_nonzero(vol.sum(axis=(1, 2))) <= len(set(d.z.tolist()))
