"""Checks of the seeded input generator (no reconstruction arithmetic here)."""
import numpy as np

from paper_1904_04884_gb300 import synth


def test_splitmix_counter_slicing_and_determinism():
    a = synth.splitmix64(42, 0, 100)
    b = synth.splitmix64(42, 37, 10)
    assert np.array_equal(a[37:47], b)
    s = synth.Stream(42)
    assert np.array_equal(np.concatenate([s.bits(30), s.bits(70)]), a)
    assert not np.array_equal(synth.splitmix64(43, 0, 100), a)


def test_splitmix_finalizer_is_a_bijection_on_samples():
    # distinct counters give distinct outputs (the mixer is invertible)
    v = synth.splitmix64(0, 0, 200000)
    assert len(np.unique(v)) == len(v)


def test_uniform_and_normal_moments():
    s = synth.Stream(7)
    u = s.uniform(200000)
    assert 0 <= u.min() and u.max() < 1
    assert abs(u.mean() - 0.5) < 3e-3 and abs(u.var() - 1 / 12) < 2e-3
    g = s.normal(200001)
    assert len(g) == 200001
    assert abs(g.mean()) < 1e-2 and abs(g.std() - 1) < 1e-2
    assert abs(((g ** 4).mean()) - 3) < 0.1


def test_disc_coverage_area():
    vol = np.zeros((1, 64, 64), np.float32)
    p = synth.Particles(np.array([32.3]), np.array([30.7]), np.array([0]), np.array([20.0]))
    synth.rasterise_discs(vol, p, supersample=8)
    assert abs(vol.sum() - np.pi * 100) / (np.pi * 100) < 0.01
    assert vol.max() == 1.0


def test_workload_volumes_are_seeded():
    from paper_1904_04884_gb300 import workloads
    a = workloads.TINY.opacity()
    b = workloads.TINY.opacity()
    assert np.array_equal(a, b)
    assert a.shape == (16, 64, 64)
    assert (a > 0).sum() > 20 * 5


def test_fibres_rasterise_inside_volume():
    vol = np.zeros((16, 64, 64), np.float32)
    synth.rasterise_fibres(vol, synth.Stream(3), 5, 50, 200, 3.0, 5.0, 25.0)
    assert vol.max() == 1.0 and vol.sum() > 5


def test_lamb_oseen_preserves_radius_and_rate():
    x0 = np.array([40.0, 10.0, 32.0])
    y0 = np.array([32.0, 32.0, 60.0])
    gam, rc = 300.0, 8.0
    x, y = synth.lamb_oseen_advect(x0, y0, gam, rc, 32.0, 32.0, frames=1.0, substeps=16)
    r0 = np.hypot(x0 - 32, y0 - 32)
    r1 = np.hypot(x - 32, y - 32)
    np.testing.assert_allclose(r1, r0, rtol=1e-6)
    ang = np.arctan2(y - 32, x - 32) - np.arctan2(y0 - 32, x0 - 32)
    ang = (ang + np.pi) % (2 * np.pi) - np.pi
    omega = gam / (2 * np.pi * r0 ** 2) * (1 - np.exp(-r0 ** 2 / rc ** 2))
    np.testing.assert_allclose(ang, omega, rtol=1e-6)
