"""Pins of the network-layer oracle: brute-force 7-loop convolution on tiny
shapes, adjoint identities, and finite differences of the weight gradient."""
import numpy as np

from oracle import unet_oracle as U


def _brute_conv(x, w, b):
    d, h, wd, cin = x.shape
    cout = w.shape[0]
    y = np.zeros((d, h, wd, cout))
    for z in range(d):
        for yy in range(h):
            for xx in range(wd):
                for o in range(cout):
                    s = b[o]
                    for t, (dz, dy, dx) in enumerate(U.OFFSETS):
                        zz, y2, x2 = z + dz, yy + dy, xx + dx
                        if 0 <= zz < d and 0 <= y2 < h and 0 <= x2 < wd:
                            for c in range(cin):
                                s += w[o, t, c] * x[zz, y2, x2, c]
                    y[z, yy, xx, o] = s
    return y


def test_conv_matches_brute_force_loops():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 4, 5, 2))
    w = rng.standard_normal((3, 27, 2))
    b = rng.standard_normal(3)
    np.testing.assert_allclose(U.conv3d(x, w, b), _brute_conv(x, w, b), atol=1e-12)


def test_tap_order_is_z_major():
    x = np.zeros((3, 3, 3, 1))
    x[2, 1, 0, 0] = 1.0               # neighbour at dz=+1, dy=0, dx=-1 of the centre
    w = np.zeros((1, 27, 1))
    t = (1 + 1) * 9 + (0 + 1) * 3 + (-1 + 1)
    w[0, t, 0] = 5.0
    assert U.conv3d(x, w)[1, 1, 1, 0] == 5.0


def test_dgrad_is_adjoint_of_conv():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((4, 5, 6, 3))
    w = rng.standard_normal((2, 27, 3))
    gy = rng.standard_normal((4, 5, 6, 2))
    lhs = np.sum(U.conv3d(x, w) * gy)
    rhs = np.sum(x * U.conv3d_dgrad(gy, w))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def test_wgrad_matches_finite_differences():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((3, 4, 4, 2))
    w = rng.standard_normal((2, 27, 2))
    gy = rng.standard_normal((3, 4, 4, 2))
    gw = U.conv3d_wgrad(x, gy)
    for (o, t, c) in [(0, 0, 0), (1, 13, 1), (0, 26, 1), (1, 5, 0)]:
        e = np.zeros_like(w)
        e[o, t, c] = 1e-6
        fd = (np.sum(U.conv3d(x, w + e) * gy) - np.sum(U.conv3d(x, w - e) * gy)) / 2e-6
        assert abs(fd - gw[o, t, c]) < 1e-6 * max(1.0, abs(fd))


def test_pool_upsample_adjoints():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((4, 6, 8, 3))
    g = rng.standard_normal((2, 3, 4, 3))
    assert abs(np.sum(U.avgpool2(x) * g) - np.sum(x * U.avgpool2_grad(g))) < 1e-12
    y = rng.standard_normal((4, 6, 8, 3))
    assert abs(np.sum(U.upsample2(g) * y) - np.sum(g * U.upsample2_grad(y))) < 1e-12
    np.testing.assert_allclose(U.avgpool2(np.ones((2, 2, 2, 1))), np.ones((1, 1, 1, 1)))


def test_relu_and_upsample_by_hand():
    """ReLU keeps positive values and zeroes the rest; nearest upsampling
    copies each voxel into its 2 x 2 x 2 cell."""
    x = np.array([-2.0, -0.0, 0.5, 3.0]).reshape(1, 1, 4, 1)
    np.testing.assert_array_equal(U.relu(x).ravel(), [0.0, 0.0, 0.5, 3.0])
    g = np.arange(2.0).reshape(1, 1, 2, 1)
    up = U.upsample2(g)
    assert up.shape == (2, 2, 4, 1)
    np.testing.assert_array_equal(up[:, :, :, 0], np.array([[[0, 0, 1, 1]] * 2] * 2))
