"""Pins of the oracle's forward model against physics and linear algebra.

Expected values come from closed forms written in wave-vector form or from the
continuous Fourier transform, not from the oracle's own formulas.
"""
import numpy as np
import pytest

from oracle import rihv_oracle as O

TINY = O.Optics(nx=32, ny=24, nz=5, wavelength=632.8e-9, pitch=10e-6, z0=5e-3, dz=100e-6)


def _plane_wave(optics, kx, ky):
    x = np.arange(optics.nx) * optics.pitch
    y = np.arange(optics.ny) * optics.pitch
    fx = kx / (optics.nx * optics.pitch)
    fy = ky / (optics.ny * optics.pitch)
    return np.exp(2j * np.pi * (fy * y[:, None] + fx * x[None, :])), fx, fy


@pytest.mark.parametrize("kx,ky", [(0, 0), (3, 0), (0, -5), (7, 4), (-16, 11), (-9, -12)])
def test_plane_wave_is_eigenfunction(kx, ky):
    """A plane wave exp(i k.r) at a grid frequency propagates by exp(i k_z z),
    k_z = sqrt(k^2 - k_x^2 - k_y^2), k = 2 pi / lambda."""
    u, fx, fy = _plane_wave(TINY, kx, ky)
    k = 2 * np.pi / TINY.wavelength
    kz = np.sqrt(k ** 2 - (2 * np.pi * fx) ** 2 - (2 * np.pi * fy) ** 2)
    z = 7.3e-3
    # The phase k_z z is ~7e4 rad; FP64 rounding of it alone is ~1e-11 rad, so
    # the bound is 64 ulp of the phase.
    atol = 64 * np.finfo(float).eps * k * z
    out = O.propagate(u, TINY, z)
    np.testing.assert_allclose(out, u * np.exp(1j * kz * z), rtol=0, atol=atol)
    # Through the volume operator: plane wave placed in plane j only.
    vol = np.zeros(TINY.shape, complex)
    vol[3] = u
    out = O.forward(vol, TINY)
    np.testing.assert_allclose(out, u * np.exp(1j * kz * (TINY.z0 + 3 * TINY.dz)), atol=atol)


def test_evanescent_components_vanish():
    """With pitch below lambda/sqrt(2) the corner frequencies are evanescent and
    are removed; propagating ones keep unit modulus."""
    op = O.Optics(nx=16, ny=16, nz=1, wavelength=632.8e-9, pitch=0.4e-6, z0=1e-6, dz=1e-6)
    u, fx, fy = _plane_wave(op, -8, -8)        # |f| = sqrt(2)/(2*0.4um) > 1/lambda
    assert op.wavelength ** 2 * (fx ** 2 + fy ** 2) > 1
    assert np.abs(O.propagate(u, op, 3e-6)).max() < 1e-13
    u2, fx2, fy2 = _plane_wave(op, 2, 1)
    np.testing.assert_allclose(np.abs(O.propagate(u2, op, 3e-6)), 1.0, atol=1e-12)


def _gaussian_setup():
    op = O.Optics(nx=128, ny=128, nz=1, wavelength=632.8e-9, pitch=10e-6, z0=0.0, dz=1e-6)
    w0 = 8 * op.pitch
    xc = 64 * op.pitch
    x = np.arange(op.nx) * op.pitch - xc
    r2 = x[None, :] ** 2 + x[:, None] ** 2
    return op, w0, x, r2


def test_gaussian_beam_paraxial_closed_form():
    """Propagated Gaussian waist matches the paraxial Gaussian beam
    u = (pi w0^2 / q) exp(-pi r^2 / q) exp(i k z), q = pi w0^2 + i lambda z,
    within the paraxial error (next term of the k_z expansion)."""
    op, w0, x, r2 = _gaussian_setup()
    u0 = np.exp(-r2 / w0 ** 2)
    for z in (5e-3, 20e-3):
        out = O.propagate(u0, op, z)
        q = np.pi * w0 ** 2 + 1j * op.wavelength * z
        ref = (np.pi * w0 ** 2 / q) * np.exp(-np.pi * r2 / q) * np.exp(2j * np.pi * z / op.wavelength)
        # paraxial phase error bound ~ 2 pi z lambda^3 f^4 / 8 at f ~ 2/(pi w0)
        f = 2.0 / (np.pi * w0)
        bound = 2 * np.pi * z * op.wavelength ** 3 * f ** 4 / 8 + 1e-12
        assert np.abs(out - ref).max() < 4 * bound, (z, np.abs(out - ref).max(), bound)


def test_gaussian_beam_direct_angular_spectrum_sum():
    """The FFT-based propagation equals the angular-spectrum integral of the
    analytic Fourier transform, summed directly in FP64 at a few points."""
    op, w0, x, r2 = _gaussian_setup()
    u0 = np.exp(-r2 / w0 ** 2)
    z = 11e-3
    out = O.propagate(u0, op, z)
    n = op.nx
    df = 1.0 / (n * op.pitch)
    f = (np.arange(n) - n // 2) * df            # symmetric band, natural order
    fy, fx = np.meshgrid(f, f, indexing="ij")
    ft = np.pi * w0 ** 2 * np.exp(-np.pi ** 2 * w0 ** 2 * (fx ** 2 + fy ** 2))
    k = 2 * np.pi / op.wavelength
    kz = np.sqrt(k ** 2 - (2 * np.pi) ** 2 * (fx ** 2 + fy ** 2))
    spec = ft * np.exp(1j * kz * z)
    for (jj, ii) in [(64, 64), (60, 71), (80, 50), (64, 90)]:
        xs, ys = x[ii], x[jj]
        val = df * df * np.sum(spec * np.exp(2j * np.pi * (fx * xs + fy * ys)))
        assert abs(val - out[jj, ii]) < 1e-11, (jj, ii, abs(val - out[jj, ii]))


def test_semigroup_and_isometry():
    rng = np.random.default_rng(1)
    u = rng.standard_normal((24, 32)) + 1j * rng.standard_normal((24, 32))
    a = O.propagate(O.propagate(u, TINY, 1.1e-3), TINY, 2.7e-3)
    b = O.propagate(u, TINY, 3.8e-3)
    np.testing.assert_allclose(a, b, atol=1e-12)
    assert abs(np.linalg.norm(O.propagate(u, TINY, 9e-3)) - np.linalg.norm(u)) < 1e-10


def test_adjoint_identity():
    """<Hx, r> = <x, H^H r> to 1e-12 relative, random complex x and r."""
    rng = np.random.default_rng(2)
    x = rng.standard_normal(TINY.shape) + 1j * rng.standard_normal(TINY.shape)
    r = rng.standard_normal((TINY.ny, TINY.nx)) + 1j * rng.standard_normal((TINY.ny, TINY.nx))
    lhs = np.vdot(r, O.forward(x, TINY))
    rhs = np.vdot(O.adjoint(r, TINY), x)
    scale = np.linalg.norm(O.forward(x, TINY)) * np.linalg.norm(r)
    assert abs(lhs - rhs) / scale < 1e-12


def test_lipschitz_matches_power_iteration():
    """2 ||H||^2 from the closed form equals 2 x the top eigenvalue of H^H H
    found by 200 power-iteration steps."""
    for op in (TINY, O.Optics(nx=16, ny=16, nz=3, wavelength=632.8e-9, pitch=0.4e-6,
                              z0=1e-6, dz=1e-6)):
        rng = np.random.default_rng(3)
        v = rng.standard_normal(op.shape) + 1j * rng.standard_normal(op.shape)
        lam = 0.0
        for _ in range(200):
            w = O.adjoint(O.forward(v, op), op)
            lam = np.linalg.norm(w) / np.linalg.norm(v)
            v = w / np.linalg.norm(w)
        assert abs(2 * lam - O.lipschitz(op)) / O.lipschitz(op) < 1e-8


def test_gradient_matches_finite_differences():
    """Re<grad f, d> equals the central difference of f = ||Hx - b||^2, which
    pins the factor 2 and the conjugation of the adjoint."""
    rng = np.random.default_rng(4)
    x = rng.standard_normal(TINY.shape) + 1j * rng.standard_normal(TINY.shape)
    d = rng.standard_normal(TINY.shape) + 1j * rng.standard_normal(TINY.shape)
    b = rng.standard_normal((TINY.ny, TINY.nx))
    eps = 1e-6
    fd = (O.data_term(x + eps * d, b, TINY) - O.data_term(x - eps * d, b, TINY)) / (2 * eps)
    an = np.vdot(O.grad_data(x, b, TINY), d).real
    assert abs(fd - an) / abs(an) < 1e-7


def test_forward_is_linear_and_sums_planes():
    rng = np.random.default_rng(5)
    x = rng.standard_normal(TINY.shape) + 1j * rng.standard_normal(TINY.shape)
    parts = []
    for j in range(TINY.nz):
        e = np.zeros_like(x)
        e[j] = x[j]
        parts.append(O.forward(e, TINY))
    np.testing.assert_allclose(sum(parts), O.forward(x, TINY), atol=1e-11)
