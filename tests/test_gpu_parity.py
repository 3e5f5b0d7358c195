"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs.

Tolerances (the parity bar of this project): relative L2 <= 1e-5 per operator
application (forward, adjoint, one fused-lasso prox call), <= 1e-3 on the final
volume after a fixed number of FISTA iterations, identical detections with
centroids within 0.5 voxel.
"""
import numpy as np
import pytest
import torch

from oracle import rihv_oracle as O
from paper_1904_04884_gb300 import synth, workloads
from paper_1904_04884_gb300.rihv import Rihv, RihvError
from tests import _detect_match as M

pytestmark = pytest.mark.gpu

OP_TOL = 1e-5
SOLVE_TOL = 1e-3


def dev():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch.device("cuda:0")


def rel_l2(a, b):
    a = np.asarray(a, np.complex128)
    b = np.asarray(b, np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex64)).to(dev())


def handle(op):
    return Rihv(op.nx, op.ny, op.nz, op.wavelength, op.pitch, op.z0, op.dz)


def optics(nx, ny, nz, wl=532e-9, pitch=5e-6, z0=5e-3, dz=50e-6):
    return O.Optics(nx=nx, ny=ny, nz=nz, wavelength=wl, pitch=pitch, z0=z0, dz=dz)


SHAPES = [(64, 48, 13), (96, 64, 7), (24, 16, 3), (768, 64, 5), (256, 256, 32), (16, 1024, 2)]


@pytest.mark.parametrize("nx,ny,nz", SHAPES)
def test_forward_parity(nx, ny, nz):
    op = optics(nx, ny, nz)
    x = synth.random_complex(synth.Stream(nx * 7 + nz), op.shape)
    h = handle(op)
    out = torch.empty((ny, nx), dtype=torch.complex64, device=dev())
    h.forward(to_dev(x), out)
    torch.cuda.synchronize()
    assert rel_l2(out.cpu().numpy(), O.forward(x, op)) <= OP_TOL


@pytest.mark.parametrize("nx,ny,nz", SHAPES)
def test_adjoint_parity(nx, ny, nz):
    op = optics(nx, ny, nz, wl=632.8e-9, pitch=10e-6, dz=100e-6)
    r = synth.random_complex(synth.Stream(nx * 11 + nz), (ny, nx))
    h = handle(op)
    out = torch.empty(op.shape, dtype=torch.complex64, device=dev())
    h.adjoint(to_dev(r), out)
    torch.cuda.synchronize()
    assert rel_l2(out.cpu().numpy(), O.adjoint(r, op)) <= OP_TOL


@pytest.mark.parametrize("rows", [1, 2, 4, 8])
@pytest.mark.parametrize("nx,ny,nz", [(128, 64, 5), (1024, 16, 2), (64, 256, 9)])
def test_row_tile_shapes_match_oracle(nx, ny, nz, rows):
    """Every row-pass tile of the register FFT engine (1, 2, 4 or 8 rows per CTA)
    gives the forward and the adjoint to the operator tolerance."""
    op = optics(nx, ny, nz)
    h = handle(op)
    h.set_options(fft_rows_per_cta=rows)
    x = synth.random_complex(synth.Stream(nx + ny + rows), op.shape)
    out = torch.empty((ny, nx), dtype=torch.complex64, device=dev())
    h.forward(to_dev(x), out)
    r = synth.random_complex(synth.Stream(nx * ny + rows), (ny, nx))
    vol = torch.empty(op.shape, dtype=torch.complex64, device=dev())
    h.adjoint(to_dev(r), vol)
    torch.cuda.synchronize()
    assert rel_l2(out.cpu().numpy(), O.forward(x, op)) <= OP_TOL
    assert rel_l2(vol.cpu().numpy(), O.adjoint(r, op)) <= OP_TOL


def test_evanescent_band_parity():
    op = optics(32, 32, 3, wl=632.8e-9, pitch=0.4e-6, z0=2e-6, dz=1e-6)
    x = synth.random_complex(synth.Stream(5), op.shape)
    h = handle(op)
    out = torch.empty((32, 32), dtype=torch.complex64, device=dev())
    h.forward(to_dev(x), out)
    torch.cuda.synchronize()
    assert rel_l2(out.cpu().numpy(), O.forward(x, op)) <= OP_TOL


def test_adjoint_identity_on_gpu():
    op = optics(128, 96, 9)
    x = synth.random_complex(synth.Stream(1), op.shape)
    r = synth.random_complex(synth.Stream(2), (op.ny, op.nx))
    h = handle(op)
    hx = torch.empty((op.ny, op.nx), dtype=torch.complex64, device=dev())
    hr = torch.empty(op.shape, dtype=torch.complex64, device=dev())
    h.forward(to_dev(x), hx)
    h.adjoint(to_dev(r), hr)
    hx, hr = hx.cpu().numpy().astype(np.complex128), hr.cpu().numpy().astype(np.complex128)
    lhs = np.vdot(r, hx)
    rhs = np.vdot(hr, x)
    assert abs(lhs - rhs) / (np.linalg.norm(hx) * np.linalg.norm(r)) < 1e-6


@pytest.mark.parametrize("per_launch", [1, 2])
@pytest.mark.parametrize("dims", [3, 2])
@pytest.mark.parametrize("nx,ny,nz,k", [(48, 24, 37, 20), (24, 16, 5, 1), (64, 32, 33, 7),
                                         (16, 16, 1, 5), (96, 48, 70, 6)])
def test_prox_parity(nx, ny, nz, k, dims, per_launch):
    op = optics(nx, ny, nz)
    v = synth.random_complex(synth.Stream(nz * 3 + k), op.shape)
    h = handle(op)
    h.set_options(tv_dims=dims, tv_steps_per_launch=per_launch)
    out = torch.empty(op.shape, dtype=torch.complex64, device=dev())
    t_l1, t_tv = 0.3, 0.05
    h.prox_fused_lasso(to_dev(v), t_l1, t_tv, k, out)
    torch.cuda.synchronize()
    ref = O.prox_fused_lasso(v, t_l1, t_tv, k, dims)
    assert rel_l2(out.cpu().numpy(), ref) <= OP_TOL


@pytest.mark.parametrize("dims", [3, 2])
@pytest.mark.parametrize("nx,ny,nz,k", [(96, 48, 37, 4), (64, 32, 5, 2), (192, 48, 33, 6)])
def test_fused_finalize_prox_matches_oracle_and_separate(nx, ny, nz, k, dims):
    """The last two-step launch forms x = soft(v - mu D^H p) itself (tile 58 x
    15, one more halo ring): same result as the separate finalize kernel and
    the oracle's prox, including ragged tiles and z-chunks."""
    op = optics(nx, ny, nz)
    v = synth.random_complex(synth.Stream(nz * 7 + k + dims), op.shape)
    h = handle(op)
    outs = {}
    for fuse in (1, 0):
        h.set_options(tv_dims=dims, tv_steps_per_launch=2, fuse_finalize=fuse)
        out = torch.empty(op.shape, dtype=torch.complex64, device=dev())
        h.prox_fused_lasso(to_dev(v), 0.3, 0.05, k, out)
        torch.cuda.synchronize()
        outs[fuse] = out.cpu().numpy()
    ref = O.prox_fused_lasso(v, 0.3, 0.05, k, dims)
    assert rel_l2(outs[1], ref) <= OP_TOL
    assert rel_l2(outs[1], outs[0]) <= OP_TOL


def test_fused_finalize_fista_matches_separate():
    """FISTA iterations with the fused finalize (x, y_{k+1}, restart product and
    the t / beta update on the device) follow the separate-kernel path."""
    op = optics(96, 64, 19)
    x_true = np.zeros(op.shape, np.complex128)
    x_true[9, 20:24, 30:34] = 1.0
    x_true[4, 40:43, 70:73] = 0.7
    b = synth.intensity_hologram(O.forward(x_true, op), 0.01, synth.Stream(5).normal(op.nx * op.ny))
    res = {}
    for fuse in (1, 0):
        h = handle(op)
        h.set_options(n_inner=6, check_every=5, tv_steps_per_launch=2, fuse_finalize=fuse)
        x = torch.empty(op.shape, dtype=torch.complex64, device=dev())
        tr = np.zeros(6)
        h.solve(b.astype(np.float32), 0.01, 0.005, 30, x, trace=tr)
        torch.cuda.synchronize()
        res[fuse] = (x.cpu().numpy(), tr)
    assert rel_l2(res[1][0], res[0][0]) <= 1e-4
    assert np.allclose(res[1][1], res[0][1], rtol=1e-5)


def test_prox_soft_threshold_only_and_identity():
    op = optics(32, 16, 4)
    v = synth.random_complex(synth.Stream(9), op.shape)
    h = handle(op)
    out = torch.empty(op.shape, dtype=torch.complex64, device=dev())
    h.prox_fused_lasso(to_dev(v), 0.7, 0.0, 20, out)
    torch.cuda.synchronize()
    assert rel_l2(out.cpu().numpy(), O.soft_threshold(v, 0.7)) <= OP_TOL
    h.prox_fused_lasso(to_dev(v), 0.0, 0.0, 0, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), v.astype(np.complex64))


def _tiny_problem():
    w = workloads.TINY
    op = O.Optics(*w.optics_tuple())
    a = w.opacity().astype(np.float64)
    b = synth.intensity_hologram(O.forward(a, op), w.sigma, w.noise())
    return w, op, b


@pytest.fixture(scope="module")
def tiny_solutions():
    w, op, b = _tiny_problem()
    x_ref, tr_ref = O.fista(b.astype(np.float64), op, w.lam_l1, w.lam_tv, w.iters, w.n_inner,
                            check_every=10)
    h = handle(op)
    x = torch.empty(op.shape, dtype=torch.complex64, device=dev())
    trace = np.zeros(w.iters // 10)
    done = h.solve(b, w.lam_l1, w.lam_tv, w.iters, x, trace=trace)
    assert done == w.iters
    return w, op, b, x.cpu().numpy(), trace, x_ref, tr_ref


def test_solve_parity_tiny(tiny_solutions):
    w, op, b, x, trace, x_ref, tr_ref = tiny_solutions
    assert rel_l2(x, x_ref) <= SOLVE_TOL
    np.testing.assert_allclose(trace, [f for _, f in tr_ref], rtol=1e-4)
    assert trace[-1] < trace[0]


def test_detection_parity_on_solutions(tiny_solutions):
    """Detections of the GPU solve match those of the oracle solve one to one
    by centroid within 0.5 voxel, with equal sizes. A component may differ
    only if it touches a voxel whose |x| is within 1e-3 max|x| of the
    threshold in either solution; the number of such exemptions is printed
    and is 0 on this workload."""
    w, op, b, x, trace, x_ref, tr_ref = tiny_solutions
    rel = 2.0 / 256.0
    h = handle(op)
    d_gpu = h.detect(to_dev(x), rel, 5)
    d_ref = O.detect(x_ref, rel, 5)
    assert len(d_ref) > 0
    band = 1e-3 * np.abs(x_ref).max()
    for min_vox in (5, 0):
        d_gpu = h.detect(to_dev(x), rel, min_vox)
        d_ref = O.detect(x_ref, rel, min_vox)
        r = M.compare(x, d_gpu, x_ref, d_ref, rel, band)
        print(f"min_vox {min_vox}: detections gpu {r['n_a']} oracle {r['n_b']} "
              f"matched {r['matched']} exempt {r['exempt']}")
        assert r["bad"] == [], r
        assert r["exempt"] <= (0 if min_vox else 2), r


def test_detection_parity_same_input():
    """Same input volume: identical components, centroids to rounding."""
    vol = workloads.TINY.opacity().astype(np.complex128)
    vol = vol + 0.002 * synth.random_complex(synth.Stream(77), vol.shape)
    op = O.Optics(*workloads.TINY.optics_tuple())
    h = handle(op)
    xd = to_dev(vol)
    d_gpu = h.detect(xd, 2.0 / 256.0, 5)
    d_ref = O.detect(vol.astype(np.complex64), 2.0 / 256.0, 5)
    assert len(d_gpu) == len(d_ref) > 0
    for g, r in zip(d_gpu, d_ref):
        assert g["first"] == r["first"] and g["nvox"] == r["nvox"]
        np.testing.assert_allclose(g["centroid"], r["centroid"], atol=1e-5)
    # min_vox = 0 keeps everything; empty volume gives nothing
    assert len(h.detect(xd, 2.0 / 256.0, 0)) >= len(d_gpu)
    assert h.detect(torch.zeros_like(xd), 2.0 / 256.0, 5) == []


def test_solve_is_deterministic_and_resumable():
    w, op, b = _tiny_problem()
    h = handle(op)
    x1 = torch.empty(op.shape, dtype=torch.complex64, device=dev())
    x2 = torch.empty_like(x1)
    h.solve(b, w.lam_l1, w.lam_tv, 12, x1)
    h.solve(b, w.lam_l1, w.lam_tv, 12, x2)
    assert torch.equal(x1, x2)
    # host output buffers and a warm start are accepted
    xh = np.zeros(op.shape, np.complex64)
    h.solve(b, w.lam_l1, w.lam_tv, 3, xh, x0=x1)
    assert np.isfinite(xh).all() and np.abs(xh).sum() > 0
    # host buffers that start inside a page (the library reads one byte of
    # every page they span before the copies) give the device result exactly
    n = int(np.prod(op.shape))
    raw = bytearray(8 * n + 4096 + 24)
    xo = np.frombuffer(raw, np.complex64, count=n, offset=24).reshape(op.shape)
    x0h = np.frombuffer(bytearray(8 * n + 40), np.complex64, count=n, offset=40).reshape(op.shape)
    x0h[...] = x1.cpu().numpy()
    xd = torch.empty_like(x1)
    h.solve(b, w.lam_l1, w.lam_tv, 3, xo, x0=x0h)
    h.solve(b, w.lam_l1, w.lam_tv, 3, xd, x0=x1)
    assert np.array_equal(xo, xd.cpu().numpy()) and np.array_equal(xo, xh)


def test_ista_single_iteration_matches_oracle():
    w, op, b = _tiny_problem()
    h = handle(op)
    h.set_options(accelerate=0, n_inner=20, check_every=0)
    x = torch.empty(op.shape, dtype=torch.complex64, device=dev())
    for iters in (1, 2, 5):
        h.solve(b, w.lam_l1, w.lam_tv, iters, x)
        ref, _ = O.fista(b.astype(np.float64), op, w.lam_l1, w.lam_tv, iters, 20, accelerate=False)
        assert rel_l2(x.cpu().numpy(), ref) <= 1e-5 * iters


def test_stop_test_ends_early():
    w, op, b = _tiny_problem()
    h = handle(op)
    x = torch.empty(op.shape, dtype=torch.complex64, device=dev())
    trace = np.zeros(5)
    h.solve(b, w.lam_l1, w.lam_tv, 50, x, trace=trace)
    h.set_options(check_every=10, f_star=float(trace[-1]), tol=1e-2)
    tr2 = np.zeros(5)
    done = h.solve(b, w.lam_l1, w.lam_tv, 50, x, trace=tr2)
    assert done < 50 and done % 10 == 0
    assert tr2[done // 10 - 1] <= trace[-1] * 1.01


def test_invalid_arguments_are_rejected():
    op = optics(32, 32, 4)
    h = handle(op)
    x = torch.zeros(op.shape, dtype=torch.complex64, device=dev())
    out = torch.zeros((32, 32), dtype=torch.complex64, device=dev())
    with pytest.raises(RihvError) as e:
        h.forward(x.data_ptr() + 8, out)        # misaligned
    assert e.value.status == 1
    host = np.zeros(op.shape, np.complex64)
    with pytest.raises(ValueError):
        h.forward(host, out)                    # the binding refuses host arrays here
    with pytest.raises(RihvError) as e:
        h.forward(host.ctypes.data, out)        # and so does the library for raw addresses
    assert e.value.status == 1
    with pytest.raises(RihvError):
        h.set_options(tv_dims=4)
    with pytest.raises(RihvError):
        h.prox_fused_lasso(x, -1.0, 0.1, 3, x)


# ---------------------------------------------------------------------------
# Full-size workload (512 x 512 x 128, the launch configuration bench.py times)
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def mid():
    w = workloads.MID
    op = O.Optics(*w.optics_tuple())
    return w, op, handle(op)


def test_full_size_forward_adjoint(mid):
    w, op, h = mid
    x = synth.random_complex(synth.Stream(101), op.shape)
    out = torch.empty((op.ny, op.nx), dtype=torch.complex64, device=dev())
    h.forward(to_dev(x), out)
    assert rel_l2(out.cpu().numpy(), O.forward(x, op)) <= OP_TOL
    r = synth.random_complex(synth.Stream(102), (op.ny, op.nx))
    vol = torch.empty(op.shape, dtype=torch.complex64, device=dev())
    h.adjoint(to_dev(r), vol)
    got = vol.cpu().numpy()
    ref = O.adjoint(r, op)
    assert rel_l2(got, ref) <= OP_TOL
    for j in (0, 63, 127):      # per-plane too
        assert rel_l2(got[j], ref[j]) <= OP_TOL


def test_full_size_prox(mid):
    w, op, h = mid
    v = synth.random_complex(synth.Stream(103), op.shape).astype(np.complex64)
    out = torch.empty(op.shape, dtype=torch.complex64, device=dev())
    h.set_options(tv_dims=3)
    # 4 dual steps: the first two-step launch (p = 0) and one reading p
    h.prox_fused_lasso(to_dev(v), 0.2, 0.05, 4, out)
    ref = O.prox_fused_lasso(v.astype(np.complex128), 0.2, 0.05, 4, 3)
    assert rel_l2(out.cpu().numpy(), ref) <= OP_TOL


@pytest.mark.parametrize("dims", [3, 2])
@pytest.mark.parametrize("nx,ny,nz", [(16, 16, 1), (24, 48, 5), (64, 32, 9), (48, 16, 3)])
def test_objective_of_the_iterate(nx, ny, nz, dims):
    """F(x_1) as the solver reports it (vectorised objective pass, four voxels
    of a row per item, ragged rows and planes at the volume faces) against the
    oracle's objective of the same x_1."""
    op = optics(nx, ny, nz)
    b = np.real(synth.random_complex(synth.Stream(nx + ny + nz), (ny, nx))).astype(np.float32)
    x0 = synth.random_complex(synth.Stream(nx * ny + nz), op.shape)
    h = handle(op)
    h.set_options(tv_dims=dims, n_inner=4, check_every=1)
    x = torch.empty(op.shape, dtype=torch.complex64, device=dev())
    tr = np.zeros(1)
    h.solve(b, 0.02, 0.01, 1, x, x0=to_dev(x0), trace=tr)
    torch.cuda.synchronize()
    xs = x.cpu().numpy().astype(np.complex128)
    ref = O.objective(xs, b.astype(np.float64), op, 0.02, 0.01, dims)
    assert abs(tr[0] - ref) <= 2e-5 * abs(ref)


@pytest.mark.parametrize("dims", [3, 2])
@pytest.mark.parametrize("nx,ny,nz", [(48, 24, 5), (96, 64, 9), (24, 48, 1)])
def test_short_solve_parity_on_ragged_grids(nx, ny, nz, dims):
    """Five FISTA iterations (momentum, restart test, objective every
    iteration) on grids with a factor 3, a single plane and ragged TV tiles,
    against the oracle's solve of the same hologram."""
    op = optics(nx, ny, nz)
    a = np.zeros(op.shape)
    a[nz // 2, ny // 3:ny // 3 + 3, nx // 4:nx // 4 + 3] = 1.0
    a[0, ny // 2:ny // 2 + 2, nx // 2:nx // 2 + 4] = 0.8
    b = synth.intensity_hologram(O.forward(a, op), 0.01, synth.Stream(nx + nz).normal(nx * ny))
    h = handle(op)
    h.set_options(tv_dims=dims, n_inner=6, check_every=1)
    x = torch.empty(op.shape, dtype=torch.complex64, device=dev())
    tr = np.zeros(5)
    h.solve(b, 0.01, 0.005, 5, x, trace=tr)
    ref, tr_ref = O.fista(b.astype(np.float64), op, 0.01, 0.005, 5, 6, dims, check_every=1)
    assert rel_l2(x.cpu().numpy(), ref) <= 1e-4
    np.testing.assert_allclose(tr, [f for _, f in tr_ref], rtol=1e-5)


@pytest.mark.parametrize("nx,ny,nz", [(128, 64, 9), (512, 32, 3), (1024, 16, 2)])
def test_solve_with_every_row_tile(nx, ny, nz):
    """Five FISTA iterations with 1, 2, 4 and 8 rows per row-pass CTA (the
    inverse row pass then runs its gradient-step epilogue in each tile
    shape): the same iterate bit for bit, and the oracle's to 1e-4."""
    op = optics(nx, ny, nz)
    a = np.zeros(op.shape)
    a[nz // 2, ny // 3:ny // 3 + 3, nx // 4:nx // 4 + 3] = 1.0
    b = synth.intensity_hologram(O.forward(a, op), 0.01, synth.Stream(nx + 3 * nz).normal(nx * ny))
    outs = []
    for rows in (1, 2, 4, 8):
        h = handle(op)
        h.set_options(n_inner=4, check_every=0, fft_rows_per_cta=rows)
        x = torch.empty(op.shape, dtype=torch.complex64, device=dev())
        h.solve(b, 0.01, 0.005, 5, x)
        outs.append(x.cpu())
        h.close()
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    ref, _ = O.fista(b.astype(np.float64), op, 0.01, 0.005, 5, 4, 3)
    assert rel_l2(outs[0].numpy(), ref) <= 1e-4
