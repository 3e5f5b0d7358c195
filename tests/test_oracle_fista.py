"""Pins of the oracle's FISTA driver: special cases with closed-form minimisers,
optimality (KKT) conditions, and ISTA's monotone descent."""
import numpy as np
import pytest

from oracle import rihv_oracle as O
from tests import _brute as B

IDENT = O.Optics(nx=16, ny=12, nz=1, wavelength=632.8e-9, pitch=10e-6, z0=0.0, dz=1e-4)
SMALL = O.Optics(nx=16, ny=16, nz=4, wavelength=632.8e-9, pitch=10e-6, z0=2e-3, dz=300e-6)


def _hologram(optics, seed):
    rng = np.random.default_rng(seed)
    a = np.zeros(optics.shape)
    for _ in range(6):
        k, j, i = (rng.integers(0, s) for s in optics.shape)
        a[k, max(j - 1, 0):j + 2, max(i - 1, 0):i + 2] = 1.0
    b = 2 * O.forward(a, optics).real + 0.01 * rng.standard_normal((optics.ny, optics.nx))
    return b


def test_identity_operator_lasso_closed_form():
    """nz = 1 at z = 0 gives H = I, so min ||x - b||^2 + lam ||x||_1 has the
    closed form x = soft_{lam/2}(b); FISTA reaches it (here in one step, since
    tau = 1/2 makes v = b)."""
    rng = np.random.default_rng(0)
    b = rng.standard_normal((IDENT.ny, IDENT.nx))
    lam = 0.6
    x, _ = O.fista(b, IDENT, lam, 0.0, iters=5, n_inner=0)
    ref = np.sign(b) * np.maximum(np.abs(b) - lam / 2, 0)
    np.testing.assert_allclose(x[0], ref, atol=1e-12)


def test_identity_operator_tv_matches_brute_force():
    """With H = I and lam_l1 = 0, the minimiser of ||x - b||^2 + lam_tv TV(x) is
    prox_{(lam_tv/2) TV}(b); compared with the certified primal-dual solve."""
    rng = np.random.default_rng(1)
    b = rng.standard_normal((IDENT.ny, IDENT.nx))
    lam_tv = 0.5
    x, _ = O.fista(b, IDENT, 0.0, lam_tv, iters=3, n_inner=3000)
    ref, gap = B.fused_lasso_prox_cp(b[None].astype(complex), lam_tv / 2, 0.0, 3,
                                     max_iter=20000, gap_tol=1e-14)
    assert np.linalg.norm(x - ref) <= np.sqrt(2 * gap) + 1e-6


def test_lasso_kkt_conditions_at_convergence():
    """After many FISTA iterations with lam_tv = 0, the subgradient optimality
    conditions of min ||Hx - b||^2 + lam ||x||_1 hold: g = 2 H^H(Hx - b) equals
    -lam x/|x| on the support and has |g| <= lam off it."""
    b = _hologram(SMALL, 2)
    lam = 0.5
    x, _ = O.fista(b, SMALL, lam, 0.0, iters=3000, n_inner=0)
    g = O.grad_data(x, b, SMALL)
    on = np.abs(x) > 1e-9
    assert on.sum() > 0
    np.testing.assert_allclose(g[on], -lam * x[on] / np.abs(x[on]), atol=2e-6)
    assert np.abs(g[~on]).max() <= lam * (1 + 1e-6)


def test_ista_monotone_without_tv():
    """ISTA with an exact prox never increases the objective. ISTA keeps no
    state between iterations (each step starts from the last iterate), so 15
    iterations in one call equal 15 chained single-iteration calls."""
    b = _hologram(SMALL, 3)
    vals = [O.objective(np.zeros(SMALL.shape), b, SMALL, 0.3, 0.0)]
    x = None
    for k in range(1, 16):
        x, _ = O.fista(b, SMALL, 0.3, 0.0, iters=1, n_inner=0, accelerate=False, x0=x)
        vals.append(O.objective(x, b, SMALL, 0.3, 0.0))
    assert all(v1 <= v0 + 1e-12 * abs(v0) for v0, v1 in zip(vals, vals[1:]))
    assert vals[-1] < vals[1] - 1e-3 * abs(vals[1])
    x15, _ = O.fista(b, SMALL, 0.3, 0.0, iters=15, n_inner=0, accelerate=False)
    np.testing.assert_array_equal(x15, x)


def test_ista_monotone_with_converged_tv_prox():
    b = _hologram(SMALL, 4)
    lam1, lamtv = 0.2, 0.3
    x = None
    vals = [O.objective(np.zeros(SMALL.shape), b, SMALL, lam1, lamtv)]
    for k in range(8):
        x, _ = O.fista(b, SMALL, lam1, lamtv, iters=1, n_inner=400, accelerate=False, x0=x)
        vals.append(O.objective(x, b, SMALL, lam1, lamtv))
    assert all(v1 <= v0 + 1e-9 * abs(v0) for v0, v1 in zip(vals, vals[1:]))


@pytest.mark.parametrize("restart", [True, False])
def test_fista_reaches_ista_fixed_point_faster(restart):
    """FISTA and many ISTA iterations approach the same minimiser (lasso case),
    and FISTA gets closer in the same number of iterations."""
    b = _hologram(SMALL, 5)
    lam = 0.4
    ref, _ = O.fista(b, SMALL, lam, 0.0, iters=4000, n_inner=0)
    xf, _ = O.fista(b, SMALL, lam, 0.0, iters=60, n_inner=0, restart=restart)
    xi, _ = O.fista(b, SMALL, lam, 0.0, iters=60, n_inner=0, accelerate=False)
    assert np.linalg.norm(xf - ref) < np.linalg.norm(xi - ref)


def test_objective_by_hand():
    """F(x) = ||Hx - b||^2 + lam_l1 ||x||_1 + lam_tv TV(x) on two coincident
    planes (H x = x_0 + x_1) with two non-zero voxels, every term by hand:
    x[0, 0, 0] = 3 + 4i and x[1, 1, 3] = -2 on a 2 x 2 x 4 grid, b = 1 at
    pixel (0, 0) and 0.5 at (1, 3). Data term |3 + 4i - 1|^2 + |-2 - 0.5|^2
    = 20 + 6.25; L1 5 + 2. TV: the first voxel has all three forward
    differences -(3 + 4i), |.| = 5 sqrt 3 (5 sqrt 2 without z); the second
    sits at the last index of every axis (Neumann: its own differences are 0)
    and enters the differences of its three predecessors along x, y and z,
    2 each (z only in 3D)."""
    op = O.Optics(nx=4, ny=2, nz=2, wavelength=632.8e-9, pitch=10e-6, z0=0.0, dz=0.0)
    x = np.zeros(op.shape, complex)
    x[0, 0, 0] = 3 + 4j
    x[1, 1, 3] = -2.0
    b = np.zeros((2, 4))
    b[0, 0] = 1.0
    b[1, 3] = 0.5
    lam1, lamtv = 0.3, 0.7
    np.testing.assert_allclose(O.data_term(x, b, op), 26.25, rtol=1e-14)
    np.testing.assert_allclose(O.objective(x, b, op, lam1, lamtv),
                               26.25 + 7 * lam1 + (5 * np.sqrt(3) + 6) * lamtv, rtol=1e-14)
    np.testing.assert_allclose(O.objective(x, b, op, lam1, lamtv, dims=2),
                               26.25 + 7 * lam1 + (5 * np.sqrt(2) + 4) * lamtv, rtol=1e-14)


def test_objective_trace_and_warm_start():
    b = _hologram(SMALL, 6)
    x, tr = O.fista(b, SMALL, 0.2, 0.1, iters=20, n_inner=10, check_every=5)
    assert [k for k, _ in tr] == [5, 10, 15, 20]
    assert tr[-1][1] < O.objective(np.zeros(SMALL.shape), b, SMALL, 0.2, 0.1)
    # Warm start from the answer of a long run barely moves.
    xl, _ = O.fista(b, SMALL, 0.2, 0.0, iters=3000, n_inner=0)
    xw, _ = O.fista(b, SMALL, 0.2, 0.0, iters=5, n_inner=0, x0=xl)
    assert np.linalg.norm(xw - xl) < 1e-6 * np.linalg.norm(xl)


@pytest.mark.parametrize("restart", [False, True])
def test_fista_iterates_match_three_sequence_form(restart):
    """The oracle's iterates x_1 ... x_30 equal those of an independent
    three-sequence statement of the same accelerated method (tests/_brute.py)
    to 1e-12, on a real operator with the TV term on. This pins the momentum
    factor (t_k - 1)/t_{k+1}, the t recurrence and, with the restart on, what
    a restart resets (t and y): the pins above look at converged or monotone
    behaviour only, where a wrong factor still passes. The trace is F at the
    iterates. The step, gradient and prox are the oracle's own, pinned
    elsewhere."""
    b = _hologram(SMALL, 7)
    lam1, lamtv, k_inner = 0.05, 0.08, 8
    tau = 1.0 / O.lipschitz(SMALL)

    def three_sequence(with_restart):
        return B.fista_three_sequence(
            lambda y: O.grad_data(y, b, SMALL),
            lambda v: O.prox_fused_lasso(v, tau * lam1, tau * lamtv, k_inner),
            tau, np.zeros(SMALL.shape), 30, restart=with_restart)

    xs = three_sequence(restart)
    # the momentum must be doing something on this problem
    assert np.linalg.norm(xs[2] - xs[1]) > 1e-6 * np.linalg.norm(xs[1])
    # and the gradient restart fires within these 30 iterations (the first
    # time at iteration 21), so what a restart resets is pinned too
    other = three_sequence(not restart)
    assert np.linalg.norm(xs[29] - other[29]) > 1e-6 * np.linalg.norm(xs[29])
    for k in (1, 2, 3, 4, 6, 9, 14, 20, 22, 25, 30):
        x, _ = O.fista(b, SMALL, lam1, lamtv, iters=k, n_inner=k_inner, restart=restart)
        ref = xs[k - 1]
        assert np.linalg.norm(x - ref) <= 1e-12 * np.linalg.norm(ref), k
    # the trace holds F at the iterates x_k (not at the extrapolated y_k)
    _, trace = O.fista(b, SMALL, lam1, lamtv, iters=30, n_inner=k_inner, restart=restart,
                       check_every=5)
    assert [k for k, _ in trace] == [5, 10, 15, 20, 25, 30]
    for k, f in trace:
        ref = O.objective(xs[k - 1], b, SMALL, lam1, lamtv)
        assert abs(f - ref) <= 1e-12 * abs(ref), k
    # and a wrong factor t_k / t_{k+1} would not agree
    ista, _ = O.fista(b, SMALL, lam1, lamtv, iters=3, n_inner=k_inner, accelerate=False)
    assert np.linalg.norm(ista - xs[2]) > 1e-6 * np.linalg.norm(xs[2])


def test_fista_iterates_by_hand():
    """Three iterations written out by hand for an operator whose algebra is
    plain: two planes both at z = 0 (nz = 2, z0 = dz = 0), so H x = x_0 + x_1,
    L = 2 ||H||^2 = 4 and tau = 1/4, and the gradient step is
    v_j = y_j - (y_0 + y_1 - b)/2 for both planes. With lam = 0 the first
    iterate from the warm start (a, 0) is ((a + b)/2, (b - a)/2). With an L1
    weight, x_k = soft_{tau lam}(v(y_k)), y_2 = x_1 (t_1 = 1) and
    y_3 = x_2 + ((t_2 - 1)/t_3)(x_2 - x_1), t_2 = (1 + sqrt 5)/2: the third
    iterate carries the momentum factor."""
    op = O.Optics(nx=4, ny=2, nz=2, wavelength=632.8e-9, pitch=10e-6, z0=0.0, dz=0.0)
    rng = np.random.default_rng(3)
    a = rng.standard_normal((2, 4))
    b = rng.standard_normal((2, 4))
    x0 = np.stack([a, np.zeros_like(a)]).astype(complex)
    x1, _ = O.fista(b, op, 0.0, 0.0, iters=1, n_inner=0, x0=x0)
    np.testing.assert_allclose(x1[0], (a + b) / 2, atol=1e-14)
    np.testing.assert_allclose(x1[1], (b - a) / 2, atol=1e-14)
    # with lam > 0: x_k = soft_{tau lam}(v_k); three iterations by hand
    lam = 0.4
    k = lam / 4.0

    def soft(u):
        return np.sign(u) * np.maximum(np.abs(u) - k, 0.0)

    def step(y):
        r = y[0] + y[1] - b
        return np.stack([soft(y[0] - r / 2), soft(y[1] - r / 2)])

    t1 = 1.0
    t2 = (1 + np.sqrt(5.0)) / 2
    t3 = (1 + np.sqrt(1 + 4 * t2 * t2)) / 2
    h1 = step(x0.real)
    y2 = h1 + (t1 - 1) / t2 * (h1 - x0.real)
    h2 = step(y2)
    y3 = h2 + (t2 - 1) / t3 * (h2 - h1)
    h3 = step(y3)
    x3, _ = O.fista(b, op, lam, 0.0, iters=3, n_inner=0, x0=x0, restart=False)
    np.testing.assert_allclose(x3.real, h3, atol=1e-13)
    assert np.abs(x3.imag).max() == 0.0
    # the momentum moved the third iterate
    assert np.abs(step(h2) - h3).max() > 1e-3


def test_fasta_on_the_identity_keeps_the_step_and_the_closed_form():
    """H = I: the gradient step with tau = 1/L = 1/2 gives v = b whatever the
    iterate, so every iterate is prox(b), dx = 0 after the first step and the
    gradient change is 2 dx: the steepest-descent and minimum-residual steps
    are both 1/2, the adaptive rule keeps 1/2 for the second step, and nothing
    backtracks. A rule off by any factor (tau_s + tau_m, tau_m / 2, ...) moves
    the second iterate away from prox(b). (At the fixed point dx = 0 and the
    rule's fallback, 1.5 times the step, takes over.)"""
    rng = np.random.default_rng(7)
    b = rng.standard_normal((IDENT.ny, IDENT.nx))
    lam1, lamtv = 0.3, 0.2
    ref = O.prox_fused_lasso(b[None].astype(complex), lam1 / 2, lamtv / 2, 200, 3)
    x1, _, info1 = O.fasta(b, IDENT, lam1, lamtv, iters=1, n_inner=200)
    np.testing.assert_allclose(x1, ref, atol=1e-13)
    x, _, info = O.fasta(b, IDENT, lam1, lamtv, iters=2, n_inner=200)
    np.testing.assert_allclose(x, ref, atol=1e-13)
    assert info["backtracks"] == 0 and np.allclose(info["taus"], [0.5, 0.5], rtol=1e-14)
    # an L1 weight that thresholds everything (lam/2 > max|b| at every step
    # s: soft_{s lam}(2 s b) = 0) keeps x = 0, so dx = 0 and the rule has no
    # curvature to go on: each step is 1.5 times the last, and with f
    # unchanged nothing backtracks
    big = 2.5 * np.abs(b).max()
    x, _, info = O.fasta(b, IDENT, big, 0.0, iters=5, n_inner=0)
    assert np.abs(x).max() == 0.0 and info["backtracks"] == 0
    np.testing.assert_allclose(info["taus"], 0.5 * 1.5 ** np.arange(5), rtol=1e-15)


def test_fasta_steps_on_two_coincident_planes_by_hand():
    """Two planes at z = 0: H x = x_0 + x_1, so H^H H x = (s, s) with
    s = x_0 + x_1, L = 2 ||H||^2 = 4. For any step, dg = 2 H^H H dx gives
    <dx, dg> = 2 ||ds||^2 and ||dg||^2 = 8 ||ds||^2 (ds = dx_0 + dx_1): the
    minimum-residual step is always 1/4 and the steepest-descent step is
    ||dx||^2 / (2 ||ds||^2). Each accepted step after the first must be 1/4
    when 1/2 > tau_s, else tau_s - 1/8 (or a backtracked fraction of it)."""
    op = O.Optics(nx=8, ny=4, nz=2, wavelength=632.8e-9, pitch=10e-6, z0=0.0, dz=0.0)
    rng = np.random.default_rng(8)
    b = rng.standard_normal((4, 8))
    x0 = rng.standard_normal((2, 4, 8)) + 1j * rng.standard_normal((2, 4, 8))
    lam = 0.3
    xs = [x0.astype(complex)]
    taus = []
    for k in range(1, 9):
        x, _, info = O.fasta(b, op, lam, 0.0, iters=k, n_inner=0, x0=x0)
        xs.append(x)
        taus = info["taus"]
    assert taus[0] == 0.25
    checked = 0
    for k in range(1, 8):
        dx = xs[k] - xs[k - 1]
        ds = dx[0] + dx[1]
        if np.vdot(ds, ds).real < 1e-12 * np.vdot(dx, dx).real:
            continue
        tau_s = np.vdot(dx, dx).real / (2 * np.vdot(ds, ds).real)
        expect = 0.25 if 0.5 > tau_s else tau_s - 0.125
        # the step used for x_{k+1} is the rule's value, or that halved by backtracking
        ratio = taus[k] / expect
        assert abs(ratio - 2.0 ** np.round(np.log2(ratio))) < 1e-9 and ratio <= 1 + 1e-12, k
        checked += 1
    assert checked >= 5 and max(taus) > 1.0      # both branches of the rule taken


def test_fasta_reaches_the_lasso_minimiser():
    """With lam_tv = 0, FASTA's limit satisfies the lasso's optimality
    conditions, like FISTA's (same problem as the KKT pin above)."""
    b = _hologram(SMALL, 2)
    lam = 0.5
    x, _, info = O.fasta(b, SMALL, lam, 0.0, iters=1500, n_inner=0)
    g = O.grad_data(x, b, SMALL)
    on = np.abs(x) > 1e-9
    assert on.sum() > 0
    np.testing.assert_allclose(g[on], -lam * x[on] / np.abs(x[on]), atol=2e-6)
    assert np.abs(g[~on]).max() <= lam * (1 + 1e-6)



def _fasta_trajectory_checked(b, optics, lam1, lamtv, k_inner, n, x0=None):
    """Run FASTA for 0 ... n iterations and check every iteration k from the
    iterates alone: x_k is the forward-backward step from x_{k-1} at the
    accepted step tau_k; that candidate meets the non-monotone test
    f(x_k) <= max of the last 10 data-term values (f(x_0) included while in
    the window) + Re<dx, g> + ||dx||^2 / (2 tau_k), within the slack of 1e-6
    of that maximum; each rejected candidate, at tau_k 2^j for j = 1 ... n_k
    (n_k halvings in iteration k), fails it; and tau_k 2^n_k is the adaptive
    step from the previous iteration's dx and dg (1/L first; the rule itself
    is worked by hand in the two-plane pin above). Returns the halvings of
    each iteration."""
    runs = [O.fasta(b, optics, lam1, lamtv, iters=k, n_inner=k_inner, x0=x0) for k in range(n + 1)]
    xs = [r[0] for r in runs]
    taus = runs[-1][2]["taus"]
    halvings = [r[2]["backtracks"] for r in runs]
    f = [O.data_term(x, b, optics) for x in xs]
    g = [O.grad_data(x, b, optics) for x in xs]

    def candidate(k, step):
        return O.prox_fused_lasso(xs[k - 1] - step * g[k - 1], step * lam1, step * lamtv, k_inner)

    def accepted(k, step, c):
        dx = c - xs[k - 1]
        f_max = max(f[max(0, k - 10):k])
        bound = f_max + np.vdot(dx, g[k - 1]).real + np.vdot(dx, dx).real / (2.0 * step)
        return O.data_term(c, b, optics) <= bound + 1e-6 * abs(f_max)

    step = 1.0 / O.lipschitz(optics)
    per = []
    for k in range(1, n + 1):
        nk = halvings[k] - halvings[k - 1]
        tk = taus[k - 1]
        assert 0 <= nk < 20
        assert abs(tk * 2.0 ** nk - step) <= 1e-12 * step, k
        np.testing.assert_allclose(xs[k], candidate(k, tk), rtol=0,
                                   atol=1e-13 * np.abs(xs[k]).max())
        assert accepted(k, tk, xs[k]), k
        for j in range(1, nk + 1):
            s = tk * 2.0 ** j
            assert not accepted(k, s, candidate(k, s)), (k, j)
        per.append(nk)
        dx, dg = xs[k] - xs[k - 1], g[k] - g[k - 1]
        dxdg = np.vdot(dx, dg).real
        if dxdg > 0:
            tau_s = np.vdot(dx, dx).real / dxdg
            tau_m = dxdg / np.vdot(dg, dg).real
            step = tau_m if 2.0 * tau_m > tau_s else tau_s - 0.5 * tau_m
        else:
            step = 1.5 * tk
    return per


def test_fasta_backtracking_meets_its_acceptance_test():
    """On a problem where FASTA backtracks often (18 halvings in 30
    iterations, several in one iteration, one candidate rejected by a margin
    of about 1e-4 of f_max), every accept and reject decision is checked
    against the non-monotone test (see the helper above). A window of another
    length, a bound without the 1/2 or with the wrong sign of Re<dx, g>, a
    slack of 1e-2 instead of 1e-6, or a halving factor other than 1/2
    changes some decision on this trajectory."""
    per = _fasta_trajectory_checked(_hologram(SMALL, 31), SMALL, 0.01, 0.005, 8, 30)
    assert sum(per) >= 15 and max(per) >= 3


def test_fasta_halves_up_to_twenty_times():
    """Two coincident planes (H x = x_0 + x_1) from a start near the null
    space (x_0 = -x_1 plus noise of the hologram's small size): the first
    steps move mostly along the null space, the steepest-descent step then
    comes out thousands of times 1/L, and the next iteration halves it 11
    times before the test accepts. A cap on halvings below 11 would take a
    candidate that fails the test."""
    op = O.Optics(nx=8, ny=4, nz=2, wavelength=632.8e-9, pitch=10e-6, z0=0.0, dz=0.0)
    rng = np.random.default_rng(12)
    a = rng.standard_normal((4, 8))
    eps = 10.0 ** rng.uniform(-4, -1)
    b = eps * rng.standard_normal((4, 8))
    x0 = np.stack([a, -a]) + eps * rng.standard_normal((2, 4, 8))
    lam = rng.uniform(0.05, 1.0)
    per = _fasta_trajectory_checked(b, op, lam, 0.0, 0, 6, x0=x0.astype(complex))
    assert max(per) == 11


def test_fasta_first_step_needs_the_rounding_slack():
    """On the identity at tau = 1/L = 1/2 the bound holds with equality in
    exact arithmetic: f(x + dx) = f(x) + Re<dx, g> + ||dx||^2 exactly for
    f = ||x - b||^2. So the first step from any start must be accepted; in
    floating point the two sides differ by rounding, and on 7 of these 40
    starts f(x_1) comes out above the bound by about 1e-17 of f. The slack
    of 1e-6 of f_max keeps all 40 from backtracking."""
    for seed in range(40):
        rng = np.random.default_rng(seed)
        b = rng.standard_normal((IDENT.ny, IDENT.nx))
        x0 = rng.standard_normal(IDENT.shape) + 1j * rng.standard_normal(IDENT.shape)
        _, _, info = O.fasta(b, IDENT, 0.3, 0.0, iters=1, n_inner=0, x0=x0)
        assert info["backtracks"] == 0 and info["taus"] == [0.5], seed
