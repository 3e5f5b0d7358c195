"""Batched solves (one CUDA graph per batch) and the autotuner."""
import os

import numpy as np
import pytest
import torch

from oracle import rihv_oracle as O
from paper_1904_04884_gb300 import synth
from paper_1904_04884_gb300.rihv import Batch, Rihv, RihvError

pytestmark = pytest.mark.gpu

SHAPES = [(64, 64, 16), (96, 64, 13), (128, 128, 24)]


def _problem(nx, ny, nz, seed):
    op = O.Optics(nx=nx, ny=ny, nz=nz, wavelength=632.8e-9, pitch=10e-6, z0=5e-3, dz=100e-6)
    a = np.zeros(op.shape)
    st = synth.Stream(seed)
    for _ in range(6):
        k, j, i = st.integers(1, nz)[0], st.integers(1, ny - 3)[0], st.integers(1, nx - 3)[0]
        a[k, j:j + 3, i:i + 3] = 1.0
    b = synth.intensity_hologram(O.forward(a, op), 0.01, synth.Stream(seed + 7).normal(nx * ny))
    return op, b


def _handle(op, **opts):
    h = Rihv(op.nx, op.ny, op.nz, op.wavelength, op.pitch, op.z0, op.dz)
    h.set_options(**opts)
    return h


def test_batch_equals_individual_solves():
    dev = torch.device("cuda:0")
    probs = [_problem(*s, seed=10 + i) for i, s in enumerate(SHAPES)]
    hs = [_handle(op, check_every=5) for op, _ in probs]
    ref = []
    ref_tr = []
    for h, (op, b) in zip(hs, probs):
        x = torch.empty(op.shape, dtype=torch.complex64, device=dev)
        tr = np.zeros(4)
        h.solve(b, 0.01, 0.005, 20, x, trace=tr)
        ref.append(x.clone())
        ref_tr.append(tr)
    batch = Batch(hs)
    for rep in range(2):                       # second call reuses the graph
        outs = [torch.empty(op.shape, dtype=torch.complex64, device=dev) for op, _ in probs]
        trs = [np.zeros(4) for _ in probs]
        batch.solve([b for _, b in probs], 0.01, 0.005, 20, outs, traces=trs)
        for o, r, t, rt in zip(outs, ref, trs, ref_tr):
            assert torch.equal(o, r)
            assert np.array_equal(t, rt)
    # warm start through the batch equals warm individual solves
    x0s = [r.clone() for r in ref]
    outs = [torch.empty_like(r) for r in ref]
    batch.solve([b for _, b in probs], 0.01, 0.005, 5, outs, x0s=x0s)
    for h, (op, b), x0, o in zip(hs, probs, x0s, outs):
        x = torch.empty_like(o)
        h.solve(b, 0.01, 0.005, 5, x, x0=x0)
        assert torch.equal(x, o)
    batch.close()


def test_batch_matches_oracle_and_host_buffers():
    probs = [_problem(*s, seed=30 + i) for i, s in enumerate(SHAPES[:2])]
    hs = [_handle(op, check_every=0, tv_steps_per_launch=2) for op, _ in probs]
    batch = Batch(hs)
    outs = [np.zeros(op.shape, np.complex64) for op, _ in probs]   # host outputs
    batch.solve([b for _, b in probs], 0.01, 0.005, 10, outs)
    for (op, b), o in zip(probs, outs):
        ref, _ = O.fista(b.astype(np.float64), op, 0.01, 0.005, 10, 20)
        assert np.linalg.norm(o - ref) / np.linalg.norm(ref) <= 1e-3
    batch.close()


def test_batch_stop_tests_inside_the_graph():
    """Handles with a stop test (f_star > 0) stop inside the batched graph at
    the same check as rihv_solve, with bitwise the same volume and trace; a
    handle without one runs all iterations; replaying the graph is stable."""
    dev = torch.device("cuda:0")
    probs = [_problem(*s, seed=50 + i) for i, s in enumerate(SHAPES)]
    f_star = []
    for op, b in probs:                       # reference objective: 60 iterations
        h = _handle(op, check_every=5)
        x = torch.empty(op.shape, dtype=torch.complex64, device=dev)
        tr = np.zeros(12)
        h.solve(b, 0.01, 0.005, 60, x, trace=tr)
        f_star.append(float(tr.min()))
    tols = [1e-2, 1e-3, None]                 # the last handle: no stop test
    hs, ref = [], []
    for (op, b), fs, tol in zip(probs, f_star, tols):
        opts = dict(check_every=5) if tol is None else dict(check_every=5, f_star=fs, tol=tol)
        h = _handle(op, **opts)
        x = torch.empty(op.shape, dtype=torch.complex64, device=dev)
        tr = np.full(8, np.nan)
        done = h.solve(b, 0.01, 0.005, 40, x, trace=tr)
        hs.append(h)
        ref.append((done, x.clone(), tr))
    assert ref[0][0] < 40 and ref[2][0] == 40
    batch = Batch(hs)
    for rep in range(2):
        outs = [torch.empty(op.shape, dtype=torch.complex64, device=dev) for op, _ in probs]
        trs = [np.zeros(8) for _ in probs]
        batch.solve([b for _, b in probs], 0.01, 0.005, 40, outs, traces=trs)
        its = batch.iterations()
        for (done, xr, trr), o, t, it in zip(ref, outs, trs, its):
            assert it == done
            assert torch.equal(o, xr)
            n = done // 5
            assert np.array_equal(t[:n], trr[:n]) and np.all(np.isnan(t[n:]))
    batch.close()


def test_batch_rejects_duplicates():
    op, b = _problem(*SHAPES[0], seed=1)
    h = _handle(op, check_every=10)
    with pytest.raises(RihvError):
        Batch([h, h])


def test_autotune_choice_is_valid_cached_and_correct(tmp_path):
    op = O.Optics(nx=96, ny=64, nz=40, wavelength=532e-9, pitch=5e-6, z0=5e-3, dz=50e-6)
    cache = str(tmp_path / "tune.txt")
    h = _handle(op)
    zc, per, zpg, rows = h.autotune(cache)
    assert zc in (8, 16, 32, 64, 128) and per in (1, 2) and 1 <= zpg <= op.nz
    assert rows == 4                                       # nx = 96: shared-memory engine
    assert os.path.exists(cache) and open(cache).read().count("rihv-tune-v2 96 64 40 3") == 1
    h2 = _handle(op)
    assert h2.autotune(cache) == (zc, per, zpg, rows)     # loaded, not searched again
    assert open(cache).read().count("rihv-tune-v2") == 1
    # the tuned handle still matches the oracle
    v = synth.random_complex(synth.Stream(5), op.shape)
    out = torch.empty(op.shape, dtype=torch.complex64, device="cuda:0")
    h2.prox_fused_lasso(torch.from_numpy(v.astype(np.complex64)).cuda(), 0.3, 0.05, 9, out)
    ref = O.prox_fused_lasso(v, 0.3, 0.05, 9)
    assert np.linalg.norm(out.cpu().numpy() - ref) / np.linalg.norm(ref) <= 1e-5
    x = synth.random_complex(synth.Stream(6), op.shape)
    y = torch.empty((op.ny, op.nx), dtype=torch.complex64, device="cuda:0")
    h2.forward(torch.from_numpy(x.astype(np.complex64)).cuda(), y)
    ref = O.forward(x, op)
    assert np.linalg.norm(y.cpu().numpy() - ref) / np.linalg.norm(ref) <= 1e-5


def test_autotune_row_tile_on_power_of_two_grid(tmp_path):
    """On a power-of-two grid the tuner also picks the row-pass tile (1, 2, 4
    or 8 rows per CTA); the tuned handle's solve matches the untuned one."""
    op = O.Optics(nx=256, ny=128, nz=24, wavelength=532e-9, pitch=5e-6, z0=5e-3, dz=50e-6)
    h = _handle(op)
    zc, per, zpg, rows = h.autotune(str(tmp_path / "tune.txt"))
    assert rows in (1, 2, 4, 8)
    x = synth.random_complex(synth.Stream(7), op.shape)
    y = torch.empty((op.ny, op.nx), dtype=torch.complex64, device="cuda:0")
    h.forward(torch.from_numpy(x.astype(np.complex64)).cuda(), y)
    ref = O.forward(x, op)
    assert np.linalg.norm(y.cpu().numpy() - ref) / np.linalg.norm(ref) <= 1e-5
