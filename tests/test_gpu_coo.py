"""Per-plane COO compaction and expansion on the GPU against the oracle's
definition (bit-exact: indices, order and values), including ragged plane
segments, empty planes and volumes, negative zeros, purely imaginary values,
the full 512 x 512 x 128 size, and argument errors."""
import numpy as np
import pytest
import torch

from oracle import rihv_oracle as O
from paper_1904_04884_gb300 import synth
from paper_1904_04884_gb300.rihv import Rihv, RihvError

pytestmark = pytest.mark.gpu


def sparse_volume(shape, density, seed):
    st = synth.Stream(seed)
    x = synth.random_complex(st, shape).astype(np.complex64)
    keep = st.uniform(int(np.prod(shape))).reshape(shape) < density
    x[~keep] = 0
    return x


def handle(shape):
    nz, ny, nx = shape
    return Rihv(nx, ny, nz, 532e-9, 5e-6, 5e-3, 50e-6)


@pytest.mark.parametrize("shape,density", [((7, 24, 48), 0.05), ((5, 64, 96), 0.3),
                                           ((1, 16, 16), 1.0), ((3, 48, 24), 0.001)])
def test_coo_compact_matches_oracle_bit_exact(shape, density):
    x = sparse_volume(shape, density, 41 + shape[0])
    x[0, 0, 0] = complex(-0.0, 0.0)             # zero
    x[-1, -1, -1] = 3j                          # purely imaginary: non-zero
    h = handle(shape)
    off, r, c, v = h.coo_compact(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    roff, rr, rc, rv = O.coo_compact(x)
    assert np.array_equal(off.cpu().numpy(), roff)
    assert np.array_equal(r.cpu().numpy(), rr)
    assert np.array_equal(c.cpu().numpy(), rc)
    assert np.array_equal(v.cpu().numpy(), rv)
    y = torch.full(shape, 7.0 + 7.0j, dtype=torch.complex64, device="cuda")
    h.coo_expand(off, r, c, v, y)
    torch.cuda.synchronize()
    assert np.array_equal(y.cpu().numpy(), x)


def test_coo_empty_volume_and_planes():
    shape = (4, 32, 48)
    h = handle(shape)
    off, r, c, v = h.coo_compact(torch.zeros(shape, dtype=torch.complex64, device="cuda"))
    assert off.cpu().tolist() == [0] * 5 and r.numel() == 0
    x = sparse_volume(shape, 0.2, 5)
    x[1] = 0
    x[3] = 0
    off, r, c, v = h.coo_compact(torch.from_numpy(x).cuda())
    roff = O.coo_compact(x)[0]
    assert np.array_equal(off.cpu().numpy(), roff) and roff[2] == roff[1] and roff[4] == roff[3]


def test_coo_full_size_512():
    shape = (128, 512, 512)
    x = sparse_volume(shape, 0.01, 77)
    h = handle(shape)
    off, r, c, v = h.coo_compact(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    roff, rr, rc, rv = O.coo_compact(x)
    assert np.array_equal(off.cpu().numpy(), roff)
    assert np.array_equal(r.cpu().numpy(), rr) and np.array_equal(c.cpu().numpy(), rc)
    assert np.array_equal(v.cpu().numpy(), rv)


def test_coo_of_the_last_solve_result():
    shape = (6, 32, 48)
    h = handle(shape)
    b = np.ones((32, 48), np.float32)
    b[10:14, 20:24] = 0.2
    x = torch.empty(shape, dtype=torch.complex64, device="cuda")
    h.solve(b, 0.05, 0.01, 10, x)
    a = h.coo_compact(None)
    e = h.coo_compact(x)
    for p, q in zip(a, e):
        assert torch.equal(p, q)


def test_coo_argument_errors():
    import ctypes
    shape = (2, 16, 16)
    h = handle(shape)
    x = torch.from_numpy(sparse_volume(shape, 0.5, 9)).cuda()
    off = torch.empty(3, dtype=torch.int64, device="cuda")
    rows = torch.empty(4, dtype=torch.int32, device="cuda")
    cols = torch.empty(4, dtype=torch.int32, device="cuda")
    vals = torch.empty(4, dtype=torch.complex64, device="cuda")
    nnz = ctypes.c_longlong()
    st = h.L.rihv_coo_compact(h.h, x.data_ptr(), off.data_ptr(), rows.data_ptr(),
                              cols.data_ptr(), vals.data_ptr(), 4, ctypes.byref(nnz))
    assert st == 1 and nnz.value == int((x != 0).sum())          # capacity too small
    # offsets that do not end at nnz, or decrease, are refused before any work
    bad = torch.tensor([0, 5, 3], dtype=torch.int64, device="cuda")
    y = torch.zeros(shape, dtype=torch.complex64, device="cuda")
    with pytest.raises(RihvError):
        h.coo_expand(bad, rows[:3], cols[:3], vals[:3], y)
    # an entry outside its plane is skipped and reported
    o2 = torch.tensor([0, 1, 1], dtype=torch.int64, device="cuda")
    r2 = torch.tensor([99], dtype=torch.int32, device="cuda")
    c2 = torch.tensor([0], dtype=torch.int32, device="cuda")
    v2 = torch.ones(1, dtype=torch.complex64, device="cuda")
    with pytest.raises(RihvError):
        h.coo_expand(o2, r2, c2, v2, y)
    assert torch.count_nonzero(y) == 0
