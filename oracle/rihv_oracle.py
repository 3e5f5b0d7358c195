"""FP64 CPU oracle for fused-lasso (L1 + TV) FISTA holographic volume reconstruction.

TEST INFRASTRUCTURE ONLY. This module exists to check the CUDA path. Only the
tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it. The product path (the ``rihv`` C-ABI library
and its Python binding) never imports, calls or links anything here, and this
module imports nothing from the product package.

Everything is plain numpy in float64 / complex128, written step by step in the
order the paper gives, so that it can be read against the paper by eye. The only
library primitives used as steps are the 2D FFT (``numpy.fft``) and connected-
component labelling (``scipy.ndimage.label``).

Paper: "Regularized Inverse Holographic Volume Reconstruction for 3D Particle
Tracking" (arXiv 1904.04884), Section 2 (Methodology).

Readings where the paper is silent or garbled:

R1  Grid and frequencies. Pixel (i, j), i fastest along x. Frequencies in FFT
    order, f_x = k_x / (n_x * pitch). Planes z_j = z0 + j*dz. (Section 2 gives no
    grid; the experiments speak of plane spacing, Section 3.2 and 3.3.)
R2  Transfer function. Angular spectrum H_z(f) = exp(i 2 pi z kappa(f)),
    kappa = sqrt(1/lambda^2 - f_x^2 - f_y^2) on the propagating band, 0 for
    evanescent frequencies. Carrier phase kept, sign +i. Periodic (unpadded) 2D
    DFT. The paper never writes H_z; it only says each plane is propagated
    forward and back (Section 2, GPU implementation paragraph).
R3  FFT convention: unnormalised forward F, inverse (1/(n_x n_y)) conj-DFT.
R4  Linearised model (Section 2, Eq. for the optimisation problem):
    H x = sum_z P_z x_z with P_z = F^-1 diag(H_z) F. The hologram b is real and
    embedded as complex; the data term is the complex ||Hx - b||^2 with no 1/2,
    so grad f = 2 H^H (Hx - b).
R5  Step size: tau = 1/L_f, L_f = 2 ||H||^2 = 2 max_f sum_z |H_z(f)|^2 (closed
    form: H H^H is diagonal in Fourier space).
R6  Soft threshold (Section 2, L1 prox equation, printed without the |v| factor):
    soft_k(u) = u * max(0, 1 - k/|u|), complex modulus; soft(0) = 0.
R7  TV (Section 2, Eq. TV_norm): isotropic first-order forward differences with
    Neumann boundary (difference 0 at the last index), extended to 3D; complex
    values are treated as R^2-valued, so |.| is the complex modulus. ``dims=2``
    drops the z difference (the paper's plane-wise 2D TV).
R8  TV prox by Beck-Teboulle gradient projection on the dual (Section 2, TV prox
    paragraph): x = v - mu D^H p, p <- Pi(p + D(v - mu D^H p) / (c mu)), with
    c = 4*dims (8 in 2D, 12 in 3D), Pi the per-voxel projection onto the unit
    ball of C^dims, p_0 = 0 at every call.
R9  Fused-lasso prox = soft threshold of the TV prox (Section 2, FL paragraph).
R10 FISTA (Beck-Teboulle 2009, as cited in Section 2) with the O'Donoghue-Candes
    gradient restart: restart when Re<y_k - x_k, x_k - x_{k-1}> > 0, which sets
    t_{k+1} = 1 and y_{k+1} = x_k. ISTA: t == 1.
R11 Detection (Section 2, last paragraphs; Section 3.2 parameters): |x| above
    rel * max|x| (strict), 26-connected components, components of <= min_vox
    voxels dropped, |x|-weighted centroid in voxel units. The threshold decision
    is taken in float32 (|x|^2 = re*re + im*im, each operation rounded to
    float32; threshold^2 = (rel*rel) * max|x|^2 in float32) so that it is the
    same decision the float32 GPU kernel takes.
R12 FASTA-style solver (Section 2 says its solver follows the FASTA
    implementation and names none of its options): forward-backward splitting x_{k+1} = prox_{tau_k g}(x_k -
    tau_k grad f(x_k)) with the adaptive spectral (Barzilai-Borwein) step of
    Goldstein, Studer and Baraniuk (steepest-descent step tau_s = <dx,dx>/<dx,dg>,
    minimum-residual step tau_m = <dx,dg>/<dg,dg>; tau = tau_m if 2 tau_m >
    tau_s, else tau_s - tau_m/2; 1.5 times the previous step when <dx,dg> <= 0)
    and their non-monotone backtracking: accept when f(x_{k+1}) <= max of the
    last 10 values of f + Re<dx, grad f(x_k)> + ||dx||^2 / (2 tau), up to a
    rounding slack of 1e-6 times that maximum (the bound is met with equality
    whenever dx lies in the top eigenspace of H^H H at tau = 1/L_f), otherwise
    halve tau and retry (at most 20 times, the last candidate then being
    taken). First step 1/L_f. Inner products
    over C^n are the real inner product of R^2n. No acceleration.
R13 Accelerated TV dual (FGP, Beck-Teboulle's fast gradient projection, the
    accelerated form of R8): p_k = Pi(r_k + D(v - mu D^H r_k)/(4 dims mu)),
    t_{k+1} = (1 + sqrt(1 + 4 t_k^2))/2, r_{k+1} = p_k + ((t_k - 1)/t_{k+1})
    (p_k - p_{k-1}), r_1 = p_0 = 0, t_1 = 1; x = v - mu D^H p_K.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


# --------------------------------------------------------------------------
# Optics and the forward model (Section 2, linearised model; readings R1-R5)
# --------------------------------------------------------------------------

@dataclass(frozen=True)
class Optics:
    """Reconstruction grid and optics. Lengths in metres."""
    nx: int
    ny: int
    nz: int
    wavelength: float
    pitch: float
    z0: float
    dz: float

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    def depths(self) -> np.ndarray:
        """Plane depths z_j = z0 + j*dz (reading R1)."""
        return self.z0 + self.dz * np.arange(self.nz, dtype=np.float64)


def frequencies(optics: Optics):
    """Spatial frequency grids (f_y, f_x) in FFT order, shape [ny][nx] (R1)."""
    fx = np.fft.fftfreq(optics.nx, d=optics.pitch)
    fy = np.fft.fftfreq(optics.ny, d=optics.pitch)
    return np.meshgrid(fy, fx, indexing="ij")


def axial_frequency(optics: Optics):
    """kappa(f) = sqrt(1/lambda^2 - f_x^2 - f_y^2) and the propagating mask (R2)."""
    fy, fx = frequencies(optics)
    arg = 1.0 / optics.wavelength ** 2 - fx ** 2 - fy ** 2
    propagating = (optics.wavelength ** 2) * (fx ** 2 + fy ** 2) < 1.0
    kappa = np.sqrt(np.where(propagating, arg, 0.0))
    return kappa, propagating


def transfer_function(optics: Optics, z: float) -> np.ndarray:
    """Angular-spectrum transfer function H_z, complex128 [ny][nx] (R2)."""
    kappa, propagating = axial_frequency(optics)
    return np.where(propagating, np.exp(2j * np.pi * z * kappa), 0.0)


def propagate(field: np.ndarray, optics: Optics, z: float) -> np.ndarray:
    """P_z u = F^-1 (H_z . F u) for one 2D field (R2, R3)."""
    return np.fft.ifft2(transfer_function(optics, z) * np.fft.fft2(field))


def forward(x: np.ndarray, optics: Optics) -> np.ndarray:
    """Modelled hologram H x = sum_z P_z x_z (Section 2, linearised model; R4).

    x: complex [nz][ny][nx]. Returns complex [ny][nx].
    """
    x = np.asarray(x, dtype=np.complex128)
    assert x.shape == optics.shape
    out = np.zeros((optics.ny, optics.nx), dtype=np.complex128)
    for j, z in enumerate(optics.depths()):
        out += propagate(x[j], optics, z)
    return out


def adjoint(r: np.ndarray, optics: Optics) -> np.ndarray:
    """H^H r = [P_z^H r]_z, P_z^H = F^-1 diag(conj H_z) F (R4).

    r: complex [ny][nx]. Returns complex [nz][ny][nx].
    """
    r = np.asarray(r, dtype=np.complex128)
    spectrum = np.fft.fft2(r)
    out = np.empty(optics.shape, dtype=np.complex128)
    for j, z in enumerate(optics.depths()):
        out[j] = np.fft.ifft2(np.conj(transfer_function(optics, z)) * spectrum)
    return out


def residual(x: np.ndarray, b: np.ndarray, optics: Optics) -> np.ndarray:
    """r = H x - b with the real hologram b embedded as complex (R4)."""
    return forward(x, optics) - np.asarray(b, dtype=np.float64)


def data_term(x: np.ndarray, b: np.ndarray, optics: Optics) -> float:
    """f(x) = ||H x - b||_2^2, no 1/2 factor (Section 2, optimisation problem)."""
    r = residual(x, b, optics)
    return float(np.vdot(r, r).real)


def grad_data(x: np.ndarray, b: np.ndarray, optics: Optics) -> np.ndarray:
    """grad f(x) = 2 H^H (H x - b) (R4)."""
    return 2.0 * adjoint(residual(x, b, optics), optics)


def lipschitz(optics: Optics) -> float:
    """L_f = 2 ||H||^2 = 2 max_f sum_z |H_z(f)|^2 (R5, closed form)."""
    acc = np.zeros((optics.ny, optics.nx))
    for z in optics.depths():
        acc += np.abs(transfer_function(optics, z)) ** 2
    return 2.0 * float(acc.max())


# --------------------------------------------------------------------------
# Regularisers (Section 2, Eqs. L1_norm, TV_norm, FL_norm; readings R6-R7)
# --------------------------------------------------------------------------

def l1_norm(x: np.ndarray) -> float:
    """||x||_1 = sum |x_i| (Section 2, Eq. L1_norm)."""
    return float(np.abs(x).sum())


def grad_op(x: np.ndarray, dims: int = 3):
    """Forward differences (D_x, D_y, D_z) with Neumann boundary (R7).

    x is [nz][ny][nx]; the difference along an axis is zero at its last index.
    For dims == 2 the z component is identically zero.
    """
    x = np.asarray(x)
    dx = np.zeros_like(x)
    dy = np.zeros_like(x)
    dzz = np.zeros_like(x)
    dx[:, :, :-1] = x[:, :, 1:] - x[:, :, :-1]
    dy[:, :-1, :] = x[:, 1:, :] - x[:, :-1, :]
    if dims == 3:
        dzz[:-1, :, :] = x[1:, :, :] - x[:-1, :, :]
    return dx, dy, dzz


def grad_op_adjoint(px, py, pz, dims: int = 3):
    """D^H p, the exact adjoint of ``grad_op`` (R7).

    (D_x^H p)_i = p_{i-1} [i >= 1] - p_i [i <= n-2]; likewise along y and z.
    """
    out = np.zeros_like(px)
    # -p_i for i <= n-2, +p_{i-1} for i >= 1
    out[:, :, :-1] -= px[:, :, :-1]
    out[:, :, 1:] += px[:, :, :-1]
    out[:, :-1, :] -= py[:, :-1, :]
    out[:, 1:, :] += py[:, :-1, :]
    if dims == 3:
        out[:-1, :, :] -= pz[:-1, :, :]
        out[1:, :, :] += pz[:-1, :, :]
    return out


def tv_norm(x: np.ndarray, dims: int = 3) -> float:
    """Isotropic TV, sum over voxels of sqrt(|D_x x|^2 + |D_y x|^2 + |D_z x|^2)
    (Section 2, Eq. TV_norm, extended to 3D; R7)."""
    dx, dy, dzz = grad_op(x, dims)
    return float(np.sqrt(np.abs(dx) ** 2 + np.abs(dy) ** 2 + np.abs(dzz) ** 2).sum())


def soft_threshold(u: np.ndarray, kappa: float) -> np.ndarray:
    """L1 prox: soft_k(u) = u * max(0, 1 - k/|u|) (Section 2, L1 prox; R6)."""
    u = np.asarray(u)
    mag = np.abs(u)
    with np.errstate(divide="ignore", invalid="ignore"):
        scale = np.where(mag > kappa, 1.0 - kappa / np.where(mag > 0, mag, 1.0), 0.0)
    return u * scale


def project_unit_ball(px, py, pz):
    """Per-voxel projection onto {|p|_2 <= 1} in C^3 (R8)."""
    norm = np.sqrt(np.abs(px) ** 2 + np.abs(py) ** 2 + np.abs(pz) ** 2)
    scale = 1.0 / np.maximum(1.0, norm)
    return px * scale, py * scale, pz * scale


def tv_prox_gp(v: np.ndarray, mu: float, n_inner: int, dims: int = 3,
               return_dual: bool = False):
    """prox_{mu TV}(v) by Beck-Teboulle dual gradient projection (Section 2, TV
    prox paragraph; R8).

    Returns x = v - mu D^H p after ``n_inner`` projected gradient steps from p = 0.
    """
    v = np.asarray(v, dtype=np.complex128)
    px = np.zeros_like(v)
    py = np.zeros_like(v)
    pz = np.zeros_like(v)
    if mu == 0.0 or n_inner == 0:
        return (v.copy(), (px, py, pz)) if return_dual else v.copy()
    step = 1.0 / (4.0 * dims * mu)
    for _ in range(n_inner):
        u = v - mu * grad_op_adjoint(px, py, pz, dims)
        gx, gy, gz = grad_op(u, dims)
        px, py, pz = project_unit_ball(px + step * gx, py + step * gy, pz + step * gz)
    x = v - mu * grad_op_adjoint(px, py, pz, dims)
    return (x, (px, py, pz)) if return_dual else x


def tv_prox_fgp(v: np.ndarray, mu: float, n_inner: int, dims: int = 3,
                return_dual: bool = False):
    """prox_{mu TV}(v) by the accelerated dual iteration (FGP; R13): the
    gradient-projection step of R8 taken at the extrapolated dual r_k."""
    v = np.asarray(v, dtype=np.complex128)
    p_prev = [np.zeros_like(v) for _ in range(3)]
    r = [np.zeros_like(v) for _ in range(3)]
    if mu == 0.0 or n_inner == 0:
        return (v.copy(), tuple(p_prev)) if return_dual else v.copy()
    step = 1.0 / (4.0 * dims * mu)
    t = 1.0
    p = p_prev
    for _ in range(n_inner):
        u = v - mu * grad_op_adjoint(*r, dims)
        gx, gy, gz = grad_op(u, dims)
        p = list(project_unit_ball(r[0] + step * gx, r[1] + step * gy, r[2] + step * gz))
        t_next = (1.0 + np.sqrt(1.0 + 4.0 * t * t)) / 2.0
        beta = (t - 1.0) / t_next
        r = [pc + beta * (pc - pp) for pc, pp in zip(p, p_prev)]
        p_prev, t = p, t_next
    x = v - mu * grad_op_adjoint(*p, dims)
    return (x, tuple(p)) if return_dual else x


def prox_fused_lasso(v: np.ndarray, t_l1: float, t_tv: float, n_inner: int,
                     dims: int = 3, fgp: bool = False) -> np.ndarray:
    """Fused-lasso prox = soft threshold of the TV prox (Section 2, FL paragraph;
    R9). ``t_l1`` and ``t_tv`` are already multiplied by the step tau. With
    ``fgp`` the TV prox runs the accelerated dual iteration (R13)."""
    tv = tv_prox_fgp if fgp else tv_prox_gp
    return soft_threshold(tv(v, t_tv, n_inner, dims), t_l1)


def objective(x: np.ndarray, b: np.ndarray, optics: Optics, lam_l1: float,
              lam_tv: float, dims: int = 3) -> float:
    """F(x) = ||Hx - b||^2 + lam_l1 ||x||_1 + lam_tv ||x||_TV (Section 2,
    optimisation problem with Eq. FL_norm)."""
    return (data_term(x, b, optics) + lam_l1 * l1_norm(x)
            + lam_tv * tv_norm(x, dims))


# --------------------------------------------------------------------------
# FISTA (Section 2, FISTA paragraph and shrinkage-step equation; R10)
# --------------------------------------------------------------------------

def fista(b: np.ndarray, optics: Optics, lam_l1: float, lam_tv: float, iters: int,
          n_inner: int, dims: int = 3, restart: bool = True,
          accelerate: bool = True, x0: np.ndarray | None = None,
          check_every: int = 0, fgp: bool = False):
    """Fused-lasso FISTA. Returns (x_final, trace) where trace lists
    (iteration, F(x_k)) every ``check_every`` iterations (and none if 0).

    Each iteration: v = y - tau grad f(y); x_k = prox_FL(v); t_{k+1} from t_k;
    y_{k+1} = x_k + ((t_k - 1)/t_{k+1}) (x_k - x_{k-1}); gradient restart.
    """
    tau = 1.0 / lipschitz(optics)
    x_prev = (np.zeros(optics.shape, np.complex128) if x0 is None
              else np.asarray(x0, np.complex128).copy())
    y = x_prev.copy()
    t = 1.0
    trace = []
    x = x_prev
    for k in range(1, iters + 1):
        v = y - tau * grad_data(y, b, optics)
        x = prox_fused_lasso(v, tau * lam_l1, tau * lam_tv, n_inner, dims, fgp)
        if accelerate:
            t_next = (1.0 + np.sqrt(1.0 + 4.0 * t * t)) / 2.0
            y_next = x + ((t - 1.0) / t_next) * (x - x_prev)
            if restart and np.vdot(x - x_prev, y - x).real > 0.0:
                t_next = 1.0
                y_next = x.copy()
        else:
            t_next = 1.0
            y_next = x.copy()
        x_prev, y, t = x, y_next, t_next
        if check_every and k % check_every == 0:
            trace.append((k, objective(x, b, optics, lam_l1, lam_tv, dims)))
    return x, trace


def fasta(b: np.ndarray, optics: Optics, lam_l1: float, lam_tv: float, iters: int,
          n_inner: int, dims: int = 3, x0: np.ndarray | None = None, window: int = 10,
          shrink: float = 0.5, max_backtracks: int = 20, fgp: bool = False,
          check_every: int = 0):
    """Forward-backward splitting with the adaptive spectral step and
    non-monotone backtracking (R12). Returns (x_final, trace, info): trace
    lists (iteration, F(x_k)) every ``check_every`` iterations; info holds the
    accepted steps tau_k and the number of backtracks."""
    tau = 1.0 / lipschitz(optics)
    x = (np.zeros(optics.shape, np.complex128) if x0 is None
         else np.asarray(x0, np.complex128).copy())
    f_hist = [data_term(x, b, optics)]
    g = grad_data(x, b, optics)
    trace, taus, backtracks = [], [], 0
    for k in range(1, iters + 1):
        for attempt in range(max_backtracks + 1):
            x_new = prox_fused_lasso(x - tau * g, tau * lam_l1, tau * lam_tv, n_inner, dims, fgp)
            dx = x_new - x
            f_new = data_term(x_new, b, optics)
            f_max = max(f_hist[-window:])
            bound = (f_max + float(np.vdot(dx, g).real)
                     + float(np.vdot(dx, dx).real) / (2.0 * tau))
            if f_new <= bound + 1e-6 * abs(f_max) or attempt == max_backtracks:
                break
            tau *= shrink
            backtracks += 1
        taus.append(tau)
        g_new = grad_data(x_new, b, optics)
        dg = g_new - g
        dxdg = float(np.vdot(dx, dg).real)
        if dxdg > 0.0:
            tau_s = float(np.vdot(dx, dx).real) / dxdg
            tau_m = dxdg / float(np.vdot(dg, dg).real)
            tau_next = tau_m if 2.0 * tau_m > tau_s else tau_s - 0.5 * tau_m
        else:
            tau_next = 0.0
        tau = tau_next if (tau_next > 0.0 and np.isfinite(tau_next)) else 1.5 * tau
        x, g = x_new, g_new
        f_hist.append(f_new)
        if check_every and k % check_every == 0:
            trace.append((k, objective(x, b, optics, lam_l1, lam_tv, dims)))
    return x, trace, {"taus": taus, "backtracks": backtracks}


# --------------------------------------------------------------------------
# Detection (Section 2, segmentation paragraph; Section 3.2 parameters; R11)
# --------------------------------------------------------------------------

def magnitude_sq_f32(x: np.ndarray) -> np.ndarray:
    """|x|^2 in float32 with each operation rounded: re*re, im*im, then the sum."""
    xr = np.ascontiguousarray(x.real, dtype=np.float32)
    xi = np.ascontiguousarray(x.imag, dtype=np.float32)
    return (xr * xr) + (xi * xi)


def detection_mask(x: np.ndarray, rel_thresh: float) -> np.ndarray:
    """Voxels with |x| > rel * max|x|, decided on float32 squares (R11)."""
    m2 = magnitude_sq_f32(x)
    rel = np.float32(rel_thresh)
    thr2 = np.float32(rel * rel) * np.float32(m2.max())
    return m2 > thr2


def detect(x: np.ndarray, rel_thresh: float = 2.0 / 256.0, min_vox: int = 5):
    """Threshold, 26-connected components, drop components of <= min_vox voxels,
    |x|-weighted centroids (R11).

    Returns a list of dicts ordered by the component's smallest linear voxel
    index, each with ``centroid`` (x, y, z) in voxel units, ``nvox``,
    ``weight`` (sum |x|) and ``first`` (the smallest linear index).
    """
    from scipy import ndimage

    mask = detection_mask(x, rel_thresh)
    labels, n = ndimage.label(mask, structure=np.ones((3, 3, 3), dtype=bool))
    if n == 0:
        return []
    w = np.abs(np.asarray(x, dtype=np.complex128))
    idx = np.nonzero(labels.ravel())[0]
    lab = labels.ravel()[idx] - 1
    kz, jy, ix = np.unravel_index(idx, labels.shape)
    wv = w.ravel()[idx]
    count = np.bincount(lab, minlength=n)
    sw = np.bincount(lab, weights=wv, minlength=n)
    sx = np.bincount(lab, weights=wv * ix, minlength=n)
    sy = np.bincount(lab, weights=wv * jy, minlength=n)
    sz = np.bincount(lab, weights=wv * kz, minlength=n)
    first = np.full(n, np.iinfo(np.int64).max)
    np.minimum.at(first, lab, idx)
    out = []
    # scipy numbers components in raster order of their first voxel, which is
    # the order of the smallest linear index.
    for c in range(n):
        if count[c] <= min_vox:
            continue
        out.append(dict(centroid=(sx[c] / sw[c], sy[c] / sw[c], sz[c] / sw[c]),
                        nvox=int(count[c]), weight=float(sw[c]),
                        first=int(first[c])))
    return out


# --------------------------------------------------------------------------
# Storage arithmetic (Section 2, GPU implementation paragraph)
# --------------------------------------------------------------------------

def dense_bytes(nvox: int) -> int:
    """Dense complex float32 storage: 8 bytes per voxel."""
    return 8 * nvox


def coo_bytes(nnz: int) -> int:
    """Per-plane COO storage: two 8-byte indices and an 8-byte complex value."""
    return 24 * nnz


def coo_break_even_sparsity() -> float:
    """Sparsity (zero fraction) above which COO storage is smaller than dense."""
    return 1.0 - 8.0 / 24.0


# --------------------------------------------------------------------------
# Per-plane COO storage (Section 2, GPU implementation paragraph)
# --------------------------------------------------------------------------

def coo_compact(x: np.ndarray):
    """Per-plane coordinate (COO) form of a volume x [nz][ny][nx]: every plane
    indexes its own non-zero elements (row j, column i, value), as the paper
    stores volumes plane by plane. Returns (plane_offsets int64 [nz+1], rows,
    cols, vals) with plane k's entries at [plane_offsets[k], plane_offsets[k+1])
    in row-major order (j, then i). An element is non-zero unless both its
    real and imaginary parts equal zero."""
    x = np.asarray(x)
    nz = x.shape[0]
    offsets = np.zeros(nz + 1, np.int64)
    rows, cols, vals = [], [], []
    for k in range(nz):
        plane = x[k]
        nzmask = (plane.real != 0) | (plane.imag != 0)
        j, i = np.nonzero(nzmask)          # row-major order
        rows.append(j)
        cols.append(i)
        vals.append(plane[j, i])
        offsets[k + 1] = offsets[k] + len(j)
    return (offsets, np.concatenate(rows).astype(np.int64), np.concatenate(cols).astype(np.int64),
            np.concatenate(vals) if vals else np.zeros(0, x.dtype))


def coo_expand(offsets, rows, cols, vals, shape, dtype=np.complex128) -> np.ndarray:
    """Dense volume from its per-plane COO form (zeros elsewhere)."""
    x = np.zeros(shape, dtype)
    for k in range(shape[0]):
        a, b = int(offsets[k]), int(offsets[k + 1])
        x[k, rows[a:b], cols[a:b]] = vals[a:b]
    return x
