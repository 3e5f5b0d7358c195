"""Independent brute-force helpers for pinning the oracle.

Nothing here calls the oracle. The difference operator is built as an explicit
sparse matrix from its definition (forward difference, zero in the last row of
each axis), and the convex problems are solved with the accelerated
primal-dual method of Chambolle and Pock (J. Math. Imaging Vis. 40, 2011,
Algorithm 2), whose duality gap certifies the answer.
"""
from __future__ import annotations

from collections import deque

import numpy as np
import scipy.sparse as sp


def diff_matrix_1d(n: int) -> sp.csr_matrix:
    """Forward difference on n points with a zero last row."""
    rows, cols, vals = [], [], []
    for i in range(n - 1):
        rows += [i, i]
        cols += [i + 1, i]
        vals += [1.0, -1.0]
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def grad_matrices(shape, dims=3):
    """(Dx, Dy, Dz) as sparse matrices acting on C-order vectors of ``shape``."""
    nz, ny, nx = shape
    ix = sp.identity(nx, format="csr")
    iy = sp.identity(ny, format="csr")
    iz = sp.identity(nz, format="csr")
    dx = sp.kron(sp.kron(iz, iy), diff_matrix_1d(nx), format="csr")
    dy = sp.kron(sp.kron(iz, diff_matrix_1d(ny)), ix, format="csr")
    if dims == 3:
        dzm = sp.kron(sp.kron(diff_matrix_1d(nz), iy), ix, format="csr")
    else:
        dzm = sp.csr_matrix((nz * ny * nx, nz * ny * nx))
    return dx, dy, dzm


def tv_iso(xv, mats):
    g = [m @ xv for m in mats]
    return float(np.sqrt(sum(np.abs(c) ** 2 for c in g)).sum())


def soft(z, k):
    mag = np.abs(z)
    with np.errstate(divide="ignore", invalid="ignore"):
        s = np.where(mag > k, 1.0 - k / np.where(mag > 0, mag, 1.0), 0.0)
    return z * s


def fused_lasso_prox_cp(v, mu, lam1=0.0, dims=3, max_iter=200000, gap_tol=1e-15):
    """argmin_x 1/2||x - v||^2 + lam1 ||x||_1 + mu TV_iso(x), by accelerated
    Chambolle-Pock. Returns (x, duality_gap)."""
    shape = v.shape
    vv = np.asarray(v, np.complex128).ravel()
    mats = grad_matrices(shape, dims)
    kop = sp.vstack(mats, format="csr")
    kh = kop.conj().T.tocsr()
    n = vv.size
    lk = 12.0 if dims == 3 else 8.0
    tau = 1.0 / np.sqrt(lk)
    sig = 1.0 / np.sqrt(lk)
    gam = 1.0
    x = vv.copy()
    xbar = x.copy()
    y = np.zeros(3 * n, np.complex128)

    def project(yy):
        c = yy.reshape(3, n)
        nrm = np.sqrt((np.abs(c) ** 2).sum(axis=0))
        return (c / np.maximum(1.0, nrm / mu)).ravel()

    def primal(xx):
        return 0.5 * np.vdot(xx - vv, xx - vv).real + lam1 * np.abs(xx).sum() + mu * tv_iso(xx, mats)

    def dual(yy):
        w = -(kh @ yy)
        xs = soft(vv + w, lam1)
        gstar = np.vdot(w, xs).real - 0.5 * np.vdot(xs - vv, xs - vv).real - lam1 * np.abs(xs).sum()
        return -gstar

    gap = np.inf
    for it in range(max_iter):
        y = project(y + sig * (kop @ xbar))
        z = x - tau * (kh @ y)
        xn = soft((z + tau * vv) / (1.0 + tau), tau * lam1 / (1.0 + tau))
        th = 1.0 / np.sqrt(1.0 + 2.0 * gam * tau)
        tau *= th
        sig /= th
        xbar = xn + th * (xn - x)
        x = xn
        if it % 200 == 199:
            gap = primal(x) - dual(y)
            if gap < gap_tol:
                break
    return x.reshape(shape), gap


def tv_prox_gap(x, p, v, mu, dims=3):
    """Duality gap P(x) - D(p) of the TV prox at primal x and dual p (|p| <= 1
    per voxel), using the sparse-matrix operator. Small gap certifies x."""
    mats = grad_matrices(v.shape, dims)
    vv = np.asarray(v, np.complex128).ravel()
    xv = np.asarray(x, np.complex128).ravel()
    px, py, pz = (np.asarray(c, np.complex128).ravel() for c in p)
    dhp = mats[0].conj().T @ px + mats[1].conj().T @ py + mats[2].conj().T @ pz
    primal = 0.5 * np.vdot(xv - vv, xv - vv).real + mu * tv_iso(xv, mats)
    dual = 0.5 * np.vdot(vv, vv).real - 0.5 * np.vdot(vv - mu * dhp, vv - mu * dhp).real
    return primal - dual


def flood_fill_components(mask):
    """26-connected components of a boolean [nz][ny][nx] mask by breadth-first
    search in raster order. Returns a list of sorted linear-index lists."""
    nz, ny, nx = mask.shape
    seen = np.zeros_like(mask, dtype=bool)
    comps = []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                if not mask[k, j, i] or seen[k, j, i]:
                    continue
                q = deque([(k, j, i)])
                seen[k, j, i] = True
                members = []
                while q:
                    a, b, c = q.popleft()
                    members.append((a * ny + b) * nx + c)
                    for da in (-1, 0, 1):
                        for db in (-1, 0, 1):
                            for dc in (-1, 0, 1):
                                aa, bb, cc = a + da, b + db, c + dc
                                if 0 <= aa < nz and 0 <= bb < ny and 0 <= cc < nx \
                                        and mask[aa, bb, cc] and not seen[aa, bb, cc]:
                                    seen[aa, bb, cc] = True
                                    q.append((aa, bb, cc))
                comps.append(sorted(members))
    return comps


def fista_three_sequence(grad, prox, tau, x0, iters, restart=False):
    """Accelerated proximal gradient in the three-sequence form (Tseng 2008,
    the form Nesterov's method is often stated in), written independently of
    the oracle's FISTA driver. With t_1 = 1, for k = 1, 2, ...:

        x_k     = prox(y_k - tau grad(y_k))
        z_k     = x_{k-1} + t_k (x_k - x_{k-1})
        t_{k+1} = the positive root of t^2 - t - t_k^2 = 0
        y_{k+1} = (1 - 1/t_{k+1}) x_k + z_k / t_{k+1}

    Expanding y_{k+1} gives Beck and Teboulle's x_k + ((t_k - 1)/t_{k+1})
    (x_k - x_{k-1}), so the iterates agree with FISTA to rounding, but every
    quantity is computed differently. With ``restart`` the gradient restart of
    O'Donoghue and Candes applies: when Re<y_k - x_k, x_k - x_{k-1}> > 0 the
    sequence starts over, t_{k+1} = 1 and y_{k+1} = x_k. ``grad`` and ``prox``
    are callables. Returns the list of iterates x_1 ... x_iters."""
    x_prev = np.array(x0, dtype=np.complex128)
    y = x_prev.copy()
    t = 1.0
    xs = []
    for _ in range(iters):
        x = prox(y - tau * grad(y))
        if restart and np.sum(((y - x).conj() * (x - x_prev)).real) > 0.0:
            t, y = 1.0, x.copy()
        else:
            z = x_prev + t * (x - x_prev)
            roots = np.roots([1.0, -1.0, -t * t])
            t = float(np.max(roots.real))
            y = (1.0 - 1.0 / t) * x + z / t
        x_prev = x
        xs.append(x)
    return xs


def project_c3(q):
    """Per-voxel projection of a stacked dual q [3][...] onto |q|_2 <= 1 in C^3."""
    nrm = np.sqrt((np.abs(q) ** 2).sum(axis=0))
    return q / np.maximum(1.0, nrm)


def tv_dual_fista(v, mu, iters, dims=3):
    """The accelerated TV dual written as plain FISTA (three-sequence form
    above) on min_q 1/2 ||v - mu D^H q||^2 over |q| <= 1, with D the sparse
    difference matrices: gradient -mu D (v - mu D^H q), step 1/(mu^2 4 dims)
    (the bound 4 dims on ||D||^2), projection as the prox. Returns the duals
    q_1 ... q_iters, each stacked [3][nz][ny][nx]."""
    shape = v.shape
    mats = grad_matrices(shape, dims)
    vv = np.asarray(v, np.complex128).ravel()

    def dh(q):
        return sum(m.conj().T @ c.ravel() for m, c in zip(mats, q))

    def grad(q):
        u = vv - mu * dh(q)
        return np.stack([-(mu * (m @ u)).reshape(shape) for m in mats])

    return fista_three_sequence(grad, project_c3, 1.0 / (mu * mu * 4.0 * dims),
                                np.zeros((3,) + shape, np.complex128), iters)
