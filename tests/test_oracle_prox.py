"""Pins of the oracle's regularisers and proximal operators.

Independent references: closed forms, sparse-matrix operators built from the
definition, and a Chambolle-Pock solve certified by its duality gap.
"""
import numpy as np
import pytest

from oracle import rihv_oracle as O
from tests import _brute as B


def _rand(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_soft_threshold_closed_forms():
    u = np.array([0.0, 3 + 4j, -2.0, 1e-3j, 0.5 * np.exp(0.3j)])
    out = O.soft_threshold(u, 0.5)
    assert out[0] == 0
    np.testing.assert_allclose(out[1], (3 + 4j) * (1 - 0.5 / 5), atol=1e-15)
    np.testing.assert_allclose(out[2], -1.5, atol=1e-15)
    assert out[3] == 0
    assert out[4] == 0                      # |u| == kappa -> exactly 0
    np.testing.assert_allclose(O.soft_threshold(u, 0.0), u)


@pytest.mark.parametrize("dims", [2, 3])
def test_difference_operator_matches_sparse_definition(dims):
    x = _rand((4, 5, 6), 1)
    mats = B.grad_matrices(x.shape, dims)
    for comp, m in zip(O.grad_op(x, dims), mats):
        np.testing.assert_allclose(comp.ravel(), m @ x.ravel(), atol=1e-14)
    p = [_rand((4, 5, 6), s) for s in (2, 3, 4)]
    dh = sum(m.conj().T @ c.ravel() for m, c in zip(mats, p))
    np.testing.assert_allclose(O.grad_op_adjoint(*p, dims).ravel(), dh, atol=1e-13)


def test_difference_operator_norm_bound():
    """||D||^2 <= 4 * dims (the constant in the gradient-projection step)."""
    for dims in (2, 3):
        mats = B.grad_matrices((6, 7, 8), dims)
        import scipy.sparse as sp
        k = sp.vstack(mats)
        smax = np.sqrt(abs(sp.linalg.eigsh((k.T @ k).astype(float), k=1)[0][0]))
        assert smax ** 2 <= 4 * dims + 1e-9


def test_tv_of_impulse():
    """Interior impulse a: the voxel itself contributes sqrt(3)|a|, each of its
    three lower neighbours |a| (forward differences)."""
    x = np.zeros((5, 5, 5), complex)
    a = 0.7 - 1.1j
    x[2, 2, 2] = a
    assert abs(O.tv_norm(x, 3) - (np.sqrt(3) + 3) * abs(a)) < 1e-14
    assert abs(O.tv_norm(x, 2) - (np.sqrt(2) + 2) * abs(a)) < 1e-14
    # At the last index the difference vanishes (Neumann): only lower neighbours.
    y = np.zeros((5, 5, 5), complex)
    y[4, 4, 4] = a
    assert abs(O.tv_norm(y, 3) - 3 * abs(a)) < 1e-14


def test_tv_prox_constant_volume_and_zero_mu():
    v = np.full((4, 5, 6), 0.3 - 0.2j)
    np.testing.assert_allclose(O.tv_prox_gp(v, 0.7, 50), v, atol=1e-15)
    w = _rand((4, 5, 6), 7)
    np.testing.assert_allclose(O.tv_prox_gp(w, 0.0, 50), w)


def test_tv_prox_step_edge_closed_form():
    """A two-plateau volume that varies along x only reduces to 1D TV: the
    plateaus move toward each other by mu/n_k along the jump direction."""
    nz, ny, nx, m = 3, 4, 10, 4
    a, c = 0.2 + 0.1j, 1.5 - 0.4j
    v = np.empty((nz, ny, nx), complex)
    v[..., :m] = a
    v[..., m:] = c
    mu = 0.3
    x = O.tv_prox_gp(v, mu, 4000)
    e = (c - a) / abs(c - a)
    np.testing.assert_allclose(x[..., :m], a + mu / m * e, atol=1e-9)
    np.testing.assert_allclose(x[..., m:], c - mu / (nx - m) * e, atol=1e-9)


@pytest.mark.parametrize("dims,shape", [(3, (4, 5, 6)), (2, (3, 6, 5)), (3, (8, 8, 8))])
def test_tv_prox_matches_chambolle_pock(dims, shape):
    """Gradient projection agrees with an independent primal-dual solve on
    volumes of 8^3 or smaller. Both answers are certified by duality gaps
    computed with the sparse-matrix operator: for the 1-strongly convex primal,
    ||x - x*|| <= sqrt(2 gap)."""
    v = _rand(shape, 11)
    mu = 0.15
    x_gp, p = O.tv_prox_gp(v, mu, 2000, dims, return_dual=True)
    gp_gap = B.tv_prox_gap(x_gp, p, v, mu, dims)
    assert gp_gap < 1e-12
    x_cp, cp_gap = B.fused_lasso_prox_cp(v, mu, 0.0, dims, max_iter=20000, gap_tol=1e-13)
    assert cp_gap < 1e-6
    bound = np.sqrt(2 * max(cp_gap, 0.0)) + np.sqrt(2 * max(gp_gap, 0.0)) + 1e-12
    assert np.linalg.norm(x_gp - x_cp) <= bound


def test_tv_prox_gap_certificate_rejects_wrong_answers():
    """The certificate is not vacuous: a perturbed or under-iterated answer
    shows a clearly positive gap."""
    v = _rand((4, 5, 6), 12)
    mu = 0.15
    x, p = O.tv_prox_gp(v, mu, 2000, 3, return_dual=True)
    assert B.tv_prox_gap(x + 1e-3, p, v, mu) > 1e-7
    x3, p3 = O.tv_prox_gp(v, mu, 3, 3, return_dual=True)
    assert B.tv_prox_gap(x3, p3, v, mu) > 1e-6


def test_fused_lasso_composition_exact_in_1d():
    """In 1D the fused-lasso prox equals the soft threshold of the TV prox
    (Friedman et al. 2007); compared with a direct primal-dual solve of the
    combined problem on real signals, within that solve's certified error."""
    rng = np.random.default_rng(5)
    for trial in range(3):
        v = rng.standard_normal((1, 1, 8)).astype(complex)
        lam1, mu = 0.3, 0.25
        x = O.prox_fused_lasso(v, lam1, mu, 20000, dims=3)
        ref, gap = B.fused_lasso_prox_cp(v, mu, lam1, 3, max_iter=60000, gap_tol=1e-14)
        assert gap < 1e-8
        assert np.linalg.norm(x - ref) <= np.sqrt(2 * gap) + 1e-9


def test_gp_is_monotone_in_dual_objective():
    """Each gradient-projection step does not increase ||v - mu D^H p||^2 (the
    dual objective), as projected gradient with step 1/L guarantees."""
    v = _rand((4, 6, 5), 21)
    mu = 0.2
    vals = []
    for k in (1, 2, 3, 5, 8, 13, 21, 34):
        x = O.tv_prox_gp(v, mu, k)
        vals.append(np.vdot(x, x).real)
    assert all(b <= a + 1e-12 for a, b in zip(vals, vals[1:]))


def _two_voxels(axis, a, c):
    """A volume of two voxels along `axis` (0 = z, 1 = y, 2 = x) holding a, c."""
    shape = [1, 1, 1]
    shape[axis] = 2
    v = np.zeros(shape, complex)
    v.reshape(-1)[:] = [a, c]
    return v


@pytest.mark.parametrize("axis", [2, 1, 0])
def test_gp_steps_by_hand(axis):
    """Gradient projection on two voxels (0, 1) one apart, worked by hand.
    From p = 0: u = v, D u = 1 on the first voxel and 0 on the last
    (Neumann), so after one step p = step = 1/(4 dims mu) there, and
    x = v - mu D^H p = (mu step, 1 - mu step) = (1/(4 dims), 1 - 1/(4 dims)):
    (1/12, 11/12) in 3D, (1/8, 7/8) in 2D at mu = 1/2. A second 3D step:
    u = (1/12, 11/12), D u = 10/12, p = 1/6 + (1/6)(10/12) = 11/36,
    x = (11/72, 61/72). Along z the 2D prox (no z difference) returns v.
    These fix the dual step constant 1/(4 dims mu), the sign and index of
    D^H, and the order of the update."""
    v = _two_voxels(axis, 0.0, 1.0)
    mu = 0.5
    x3 = O.tv_prox_gp(v, mu, 1, dims=3).reshape(-1)
    np.testing.assert_allclose(x3, [1 / 12, 11 / 12], atol=1e-15)
    x3b = O.tv_prox_gp(v, mu, 2, dims=3).reshape(-1)
    np.testing.assert_allclose(x3b, [11 / 72, 61 / 72], atol=1e-15)
    x2 = O.tv_prox_gp(v, mu, 1, dims=2).reshape(-1)
    if axis == 0:
        np.testing.assert_allclose(x2, [0.0, 1.0], atol=0)
    else:
        np.testing.assert_allclose(x2, [1 / 8, 7 / 8], atol=1e-15)
    # complex values: the same numbers along the imaginary axis
    xi = O.tv_prox_gp(_two_voxels(axis, 0.0, 1j), mu, 1, dims=3).reshape(-1)
    np.testing.assert_allclose(xi, [1j / 12, 11j / 12], atol=1e-15)


def test_gp_projection_by_hand():
    """A jump of 10 at mu = 1/2: step * D u = 10/6 > 1, so the projection
    clips p to 1 and x = (mu, 10 - mu) = (0.5, 9.5). With two components
    (a jump of 3 along x and 4 along y from the corner voxel of a 2 x 2
    plane), the corner's dual (3, 4)/6 has norm 5/6 < 1 and is kept; a jump
    of (6, 8) gives (1, 4/3), norm 5/3, scaled back to (0.6, 0.8)."""
    v = _two_voxels(2, 0.0, 10.0)
    np.testing.assert_allclose(O.tv_prox_gp(v, 0.5, 1, 3).reshape(-1), [0.5, 9.5], atol=1e-14)
    for jx, jy, pxy in ((3.0, 4.0, (0.5, 2 / 3)), (6.0, 8.0, (0.6, 0.8))):
        w = np.zeros((1, 2, 2), complex)
        w[0, 0, 1] = jx
        w[0, 1, 0] = jy
        x, (px, py, pz) = O.tv_prox_gp(w, 0.5, 1, 3, return_dual=True)
        np.testing.assert_allclose([px[0, 0, 0].real, py[0, 0, 0].real], pxy, atol=1e-14)
        # the corner has no backward neighbours: D^H p there is -(p_x + p_y)
        dh00 = -(px[0, 0, 0] + py[0, 0, 0])
        np.testing.assert_allclose(x[0, 0, 0], w[0, 0, 0] - 0.5 * dh00, atol=1e-14)


@pytest.mark.parametrize("dims", [3, 2])
def test_fgp_duals_match_plain_fista_on_the_dual(dims):
    """The oracle's accelerated dual iteration (FGP) equals FISTA, written
    independently in three-sequence form with sparse-matrix operators, applied
    to the TV dual problem: the duals after 1, 2, 5 and 12 steps to 1e-12,
    and the resulting prox."""
    v = _rand((4, 6, 5), 31)
    mu = 0.2
    qs = B.tv_dual_fista(v, mu, 12, dims)
    for k in (1, 2, 5, 12):
        x, p = O.tv_prox_fgp(v, mu, k, dims, return_dual=True)
        q = qs[k - 1]
        for c in range(3 if dims == 3 else 2):
            np.testing.assert_allclose(p[c], q[c], atol=1e-12)
    # acceleration changes the iterates from the plain gradient projection
    assert np.linalg.norm(O.tv_prox_fgp(v, mu, 5, dims) - O.tv_prox_gp(v, mu, 5, dims)) > 1e-6


def test_fgp_converges_to_the_certified_prox():
    v = _rand((4, 5, 6), 32)
    mu = 0.15
    x, p = O.tv_prox_fgp(v, mu, 3000, 3, return_dual=True)
    assert B.tv_prox_gap(x, p, v, mu) < 1e-12
    x_gp = O.tv_prox_gp(v, mu, 6000, 3)
    assert np.linalg.norm(x - x_gp) < 1e-6 * np.linalg.norm(x)
