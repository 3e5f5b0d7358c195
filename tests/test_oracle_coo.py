"""Pins of the oracle's per-plane COO form (Section 2, GPU implementation
paragraph: each plane indexes its own non-zero elements)."""
import numpy as np

from oracle import rihv_oracle as O


def test_coo_hand_example():
    # 2 planes of 3 x 4: entries written out by hand from the definition
    x = np.zeros((2, 3, 4), np.complex64)
    x[0, 0, 3] = 1 + 2j
    x[0, 2, 1] = -3j
    x[1, 1, 0] = 0.5
    x[1, 1, 2] = -0.0 + 0j       # a negative zero is zero
    x[1, 2, 3] = 2 - 1j
    off, r, c, v = O.coo_compact(x)
    assert off.tolist() == [0, 2, 4]
    assert r.tolist() == [0, 2, 1, 2]
    assert c.tolist() == [3, 1, 0, 3]
    assert v.tolist() == [1 + 2j, -3j, 0.5, 2 - 1j]


def test_coo_round_trip_and_order():
    rng = np.random.default_rng(3)
    x = (rng.normal(size=(5, 7, 9)) + 1j * rng.normal(size=(5, 7, 9))).astype(np.complex64)
    x[rng.random(x.shape) < 0.8] = 0
    x[2] = 0                                  # an empty plane
    x[3, 1, 1] = 1j                           # purely imaginary counts as non-zero
    off, r, c, v = O.coo_compact(x)
    assert off[-1] == np.count_nonzero(x)
    assert off[3] == off[2]                   # the empty plane
    for k in range(5):
        key = r[off[k]:off[k + 1]] * 9 + c[off[k]:off[k + 1]]
        assert np.all(np.diff(key) > 0)       # row-major, no duplicates
    y = O.coo_expand(off, r, c, v, x.shape, np.complex64)
    assert np.array_equal(y, x)


def test_coo_empty_and_full():
    z = np.zeros((3, 4, 4), np.complex64)
    off, r, c, v = O.coo_compact(z)
    assert off.tolist() == [0, 0, 0, 0] and len(r) == len(c) == len(v) == 0
    f = np.ones((2, 2, 3), np.complex64)
    off, r, c, v = O.coo_compact(f)
    assert off.tolist() == [0, 6, 12]
    assert r.tolist() == [0, 0, 0, 1, 1, 1] * 2 and c.tolist() == [0, 1, 2] * 4
