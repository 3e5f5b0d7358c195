"""The accelerated TV dual (FGP, option tv_fgp) and the FASTA-style solver
(option solver = 1) through the C ABI against the FP64 oracle's versions:
the prox to the operator tolerance, FISTA with the FGP prox, and FASTA's
iterates, objective trace, accepted steps and backtracks."""
import numpy as np
import pytest
import torch

from oracle import rihv_oracle as O
from paper_1904_04884_gb300 import synth, workloads
from paper_1904_04884_gb300.rihv import Batch, Rihv, RihvError

pytestmark = pytest.mark.gpu

OP_TOL = 1e-5


def rel_l2(a, b):
    a = np.asarray(a, np.complex128)
    b = np.asarray(b, np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def optics(nx, ny, nz, wl=532e-9, pitch=5e-6, z0=5e-3, dz=50e-6):
    return O.Optics(nx=nx, ny=ny, nz=nz, wavelength=wl, pitch=pitch, z0=z0, dz=dz)


def handle(op, **opts):
    h = Rihv(op.nx, op.ny, op.nz, op.wavelength, op.pitch, op.z0, op.dz)
    if opts:
        h.set_options(**opts)
    return h


@pytest.mark.parametrize("dims", [3, 2])
@pytest.mark.parametrize("nx,ny,nz,k", [(48, 24, 37, 20), (24, 16, 5, 1), (64, 32, 33, 7),
                                         (16, 16, 1, 2), (96, 48, 70, 6)])
def test_fgp_prox_matches_oracle(nx, ny, nz, k, dims):
    op = optics(nx, ny, nz)
    v = synth.random_complex(synth.Stream(nz * 5 + k + dims), op.shape)
    h = handle(op, tv_dims=dims, tv_fgp=1)
    out = torch.empty(op.shape, dtype=torch.complex64, device="cuda:0")
    h.prox_fused_lasso(torch.from_numpy(v.astype(np.complex64)).cuda(), 0.3, 0.5, k, out)
    torch.cuda.synchronize()
    ref = O.prox_fused_lasso(v, 0.3, 0.5, k, dims, fgp=True)
    assert rel_l2(out.cpu().numpy(), ref) <= OP_TOL
    if k > 2:      # from the third step on, the accelerated dual differs from the plain one
        assert rel_l2(ref, O.prox_fused_lasso(v, 0.3, 0.5, k, dims)) > 100 * OP_TOL


def _tiny():
    w = workloads.TINY
    op = O.Optics(*w.optics_tuple())
    b = synth.intensity_hologram(O.forward(w.opacity().astype(np.float64), op), w.sigma,
                                 w.noise())
    return w, op, b


def test_fista_with_fgp_prox_matches_oracle():
    w, op, b = _tiny()
    h = handle(op, n_inner=w.n_inner, check_every=5, tv_fgp=1)
    x = torch.empty(op.shape, dtype=torch.complex64, device="cuda:0")
    tr = np.zeros(4)
    h.solve(b, w.lam_l1, w.lam_tv, 20, x, trace=tr)
    ref, tr_ref = O.fista(b.astype(np.float64), op, w.lam_l1, w.lam_tv, 20, w.n_inner,
                          check_every=5, fgp=True)
    assert rel_l2(x.cpu().numpy(), ref) <= 1e-3
    np.testing.assert_allclose(tr, [f for _, f in tr_ref], rtol=1e-4)


@pytest.mark.parametrize("lam_tv,iters", [(0.005, 12), (0.0, 25)])
def test_fasta_matches_oracle(lam_tv, iters):
    """Same iterates, objective trace, accepted steps and backtracks as the
    oracle's FASTA-style solver (decisions taken on FP64 sums on both sides)."""
    w, op, b = _tiny()
    h = handle(op, n_inner=w.n_inner, check_every=4, solver=1)
    x = torch.empty(op.shape, dtype=torch.complex64, device="cuda:0")
    tr = np.zeros(iters // 4)
    done = h.solve(b, w.lam_l1, lam_tv, iters, x, trace=tr)
    assert done == iters
    taus, backtracks = h.fasta_steps()
    ref, tr_ref, info = O.fasta(b.astype(np.float64), op, w.lam_l1, lam_tv, iters, w.n_inner,
                                check_every=4)
    print(f"lam_tv {lam_tv}: backtracks {backtracks} (oracle {info['backtracks']}), "
          f"steps {np.round(taus, 6).tolist()}")
    assert backtracks == info["backtracks"]
    np.testing.assert_allclose(taus, info["taus"], rtol=1e-3)
    assert rel_l2(x.cpu().numpy(), ref) <= 1e-3
    np.testing.assert_allclose(tr, [f for _, f in tr_ref], rtol=1e-4)


def test_fasta_stop_test_and_batch_refusal():
    w, op, b = _tiny()
    h = handle(op, n_inner=w.n_inner, check_every=5, solver=1)
    x = torch.empty(op.shape, dtype=torch.complex64, device="cuda:0")
    tr = np.zeros(8)
    h.solve(b, w.lam_l1, w.lam_tv, 40, x, trace=tr)
    # the method is not monotone (the objective jumps after long steps), so the
    # stop threshold is 10 % above the last value: met first at iteration 10
    h.set_options(n_inner=w.n_inner, check_every=5, solver=1, f_star=float(tr[-1]), tol=0.1)
    tr2 = np.zeros(8)
    done = h.solve(b, w.lam_l1, w.lam_tv, 40, x, trace=tr2)
    first = next(5 * (i + 1) for i, f in enumerate(tr) if f <= tr[-1] * 1.1)
    assert done == first < 40 and tr2[done // 5 - 1] <= tr[-1] * 1.1
    with pytest.raises(RihvError):
        Batch([h]).solve([b], w.lam_l1, w.lam_tv, 10, [x])


@pytest.mark.parametrize("warm", [False, True])
def test_fasta_between_batched_solves(warm):
    """A FASTA solve ends with x in whichever of its two buffers took the last
    accepted step; a batched graph captured before it must still find its
    input and its result where it left them. The batch's results before and
    after a FASTA solve of an odd number of iterations on the same handle
    agree bit for bit."""
    w, op, b = _tiny()
    h = handle(op, n_inner=w.n_inner, check_every=0)
    bt = Batch([h])
    x0 = [torch.from_numpy(0.1 * synth.random_complex(synth.Stream(77), op.shape)
                           .astype(np.complex64)).cuda()] if warm else None
    x1 = torch.empty(op.shape, dtype=torch.complex64, device="cuda:0")
    bt.solve([b], w.lam_l1, w.lam_tv, 10, [x1], x0s=x0)
    h.set_options(n_inner=w.n_inner, check_every=0, solver=1)
    xf = torch.empty_like(x1)
    h.solve(b, w.lam_l1, w.lam_tv, 7, xf)
    same_parts = [(d["first"], d["nvox"]) for d in h.detect(xf)]
    assert [(d["first"], d["nvox"]) for d in h.detect(None)] == same_parts
    h.set_options(n_inner=w.n_inner, check_every=0)
    x2 = torch.empty_like(x1)
    bt.solve([b], w.lam_l1, w.lam_tv, 10, [x2], x0s=x0)
    assert torch.equal(x1, x2)
    assert not torch.equal(x1, xf)
