"""Mutation check of the oracle's pins (run by hand, not collected by pytest).

Each mutant is one plausible mistake planted in a copy of the oracle: a
dropped term, a wrong sign or index, a transposed operand, a wrong constant
or default. For every mutant the oracle is copied with the tests into a
temporary directory, the mistake is written into the copy, and the oracle's
CPU pins are run there; a mutant is killed when a pin fails. The repository
itself is never modified.

Expected result: every mutant is killed except "soft tie" (> against >= in
the soft threshold), which is equivalent: at |u| = k both forms give 0.

Usage:  python tests/oracle_mutants.py [-j JOBS] [NAME_FRAGMENT ...]
"""
from __future__ import annotations

import argparse
import os
import shutil
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CORE_TESTS = ["tests/test_oracle_optics.py", "tests/test_oracle_prox.py",
              "tests/test_oracle_fista.py", "tests/test_oracle_detect.py",
              "tests/test_oracle_coo.py", "tests/test_paper_values.py",
              "tests/test_detect_match.py"]
UNET_TESTS = ["tests/test_oracle_unet.py"]
EQUIVALENT = {"soft tie"}

# (name, text in the oracle, its replacement)
CORE = [
 ("arg sign fy", "- fx ** 2 - fy ** 2", "- fx ** 2 + fy ** 2"),
 ("H sign", "np.exp(2j * np.pi * z * kappa)", "np.exp(-2j * np.pi * z * kappa)"),
 ("H 2pi->pi", "np.exp(2j * np.pi * z * kappa)", "np.exp(1j * np.pi * z * kappa)"),
 ("depth offset", "self.z0 + self.dz * np.arange(self.nz, dtype=np.float64)", "self.z0 + self.dz * (1 + np.arange(self.nz, dtype=np.float64))"),
 ("adjoint no conj", "np.conj(transfer_function(optics, z)) * spectrum", "transfer_function(optics, z) * spectrum"),
 ("residual sign", "return forward(x, optics) - np.asarray(b, dtype=np.float64)", "return np.asarray(b, dtype=np.float64) - forward(x, optics)"),
 ("grad factor", "return 2.0 * adjoint(residual", "return 1.0 * adjoint(residual"),
 ("lipschitz factor", "return 2.0 * float(acc.max())", "return 1.0 * float(acc.max())"),
 ("lipschitz mean", "return 2.0 * float(acc.max())", "return 2.0 * float(acc.mean())"),
 ("l1 real", "float(np.abs(x).sum())", "float(np.abs(x.real).sum())"),
 ("Dx sign", "dx[:, :, :-1] = x[:, :, 1:] - x[:, :, :-1]", "dx[:, :, :-1] = x[:, :, :-1] - x[:, :, 1:]"),
 ("Dz off", "    if dims == 3:\n        dzz[:-1", "    if dims == 4:\n        dzz[:-1"),
 ("DH x index", "out[:, :, 1:] += px[:, :, :-1]", "out[:, :, 1:] += px[:, :, 1:]"),
 ("DH y sign", "out[:, 1:, :] += py[:, :-1, :]", "out[:, 1:, :] -= py[:, :-1, :]"),
 ("DH z off", "    if dims == 3:\n        out[:-1", "    if dims == 4:\n        out[:-1"),
 ("tv aniso", "np.sqrt(np.abs(dx) ** 2 + np.abs(dy) ** 2 + np.abs(dzz) ** 2).sum()", "(np.abs(dx) + np.abs(dy) + np.abs(dzz)).sum()"),
 ("soft tie", "np.where(mag > kappa, 1.0", "np.where(mag >= kappa, 1.0"),
 ("soft half", "1.0 - kappa / np.where", "1.0 - 0.5 * kappa / np.where"),
 ("proj sq", "scale = 1.0 / np.maximum(1.0, norm)", "scale = 1.0 / np.maximum(1.0, norm ** 2)"),
 ("proj no z", "np.abs(px) ** 2 + np.abs(py) ** 2 + np.abs(pz) ** 2)\n    scale", "np.abs(px) ** 2 + np.abs(py) ** 2)\n    scale"),
 ("gp step 8", "    step = 1.0 / (4.0 * dims * mu)\n    for _ in range(n_inner):\n        u", "    step = 1.0 / (8.0 * dims * mu)\n    for _ in range(n_inner):\n        u"),
 ("gp u sign", "        u = v - mu * grad_op_adjoint(px, py, pz, dims)", "        u = v + mu * grad_op_adjoint(px, py, pz, dims)"),
 ("gp final half", "    x = v - mu * grad_op_adjoint(px, py, pz, dims)\n    return (x, (px, py, pz))", "    x = v - 0.5 * mu * grad_op_adjoint(px, py, pz, dims)\n    return (x, (px, py, pz))"),
 ("fgp beta", "        beta = (t - 1.0) / t_next\n        r = ", "        beta = t / t_next\n        r = "),
 ("fgp extrap sign", "r = [pc + beta * (pc - pp)", "r = [pc + beta * (pp - pc)"),
 ("fgp step at p", "project_unit_ball(r[0] + step * gx, r[1] + step * gy, r[2] + step * gz)", "project_unit_ball(p_prev[0] + step * gx, p_prev[1] + step * gy, p_prev[2] + step * gz)"),
 ("fgp step 8", "    step = 1.0 / (4.0 * dims * mu)\n    t = 1.0", "    step = 1.0 / (8.0 * dims * mu)\n    t = 1.0"),
 ("fgp t 2", "        t_next = (1.0 + np.sqrt(1.0 + 4.0 * t * t)) / 2.0\n        beta", "        t_next = (1.0 + np.sqrt(1.0 + 2.0 * t * t)) / 2.0\n        beta"),
 ("fl order", "return soft_threshold(tv(v, t_tv, n_inner, dims), t_l1)", "return tv(soft_threshold(v, t_l1), t_tv, n_inner, dims)"),
 ("objective dims", "+ lam_tv * tv_norm(x, dims))", "+ lam_tv * tv_norm(x, 3))"),
 ("objective l1 half", "(data_term(x, b, optics) + lam_l1 * l1_norm(x)", "(data_term(x, b, optics) + 0.5 * lam_l1 * l1_norm(x)"),
 ("fista momentum", "y_next = x + ((t - 1.0) / t_next) * (x - x_prev)", "y_next = x + (t / t_next) * (x - x_prev)"),
 ("fista restart sign", "np.vdot(x - x_prev, y - x).real > 0.0", "np.vdot(x - x_prev, y - x).real < 0.0"),
 ("fista restart arg", "np.vdot(x - x_prev, y - x).real > 0.0", "np.vdot(x - x_prev, x - y).real > 0.0"),
 ("fista t 2", "            t_next = (1.0 + np.sqrt(1.0 + 4.0 * t * t)) / 2.0\n            y_next", "            t_next = (1.0 + np.sqrt(1.0 + 2.0 * t * t)) / 2.0\n            y_next"),
 ("fista restart keeps y", "                t_next = 1.0\n                y_next = x.copy()", "                t_next = 1.0"),
 ("fista restart keeps t", "                t_next = 1.0\n                y_next = x.copy()", "                y_next = x.copy()"),
 ("fista grad at x_prev", "v = y - tau * grad_data(y, b, optics)", "v = y - tau * grad_data(x_prev, b, optics)"),
 ("fista trace at y", "trace.append((k, objective(x, b, optics, lam_l1, lam_tv, dims)))\n    return x, trace\n", "trace.append((k, objective(y, b, optics, lam_l1, lam_tv, dims)))\n    return x, trace\n"),
 ("fista tau half", "    tau = 1.0 / lipschitz(optics)\n    x_prev", "    tau = 0.5 / lipschitz(optics)\n    x_prev"),
 ("fista x0 ignored", "    x_prev = (np.zeros(optics.shape, np.complex128) if x0 is None\n              else np.asarray(x0, np.complex128).copy())", "    x_prev = np.zeros(optics.shape, np.complex128)"),
 ("fasta window all", "f_max = max(f_hist[-window:])", "f_max = max(f_hist)"),
 ("fasta window last", "f_max = max(f_hist[-window:])", "f_max = f_hist[-1]"),
 ("fasta bound tau", "float(np.vdot(dx, dx).real) / (2.0 * tau))", "float(np.vdot(dx, dx).real) / tau)"),
 ("fasta bound sign", "bound = (f_max + float(np.vdot(dx, g).real)", "bound = (f_max - float(np.vdot(dx, g).real)"),
 ("fasta rule", "tau_next = tau_m if 2.0 * tau_m > tau_s else", "tau_next = tau_m if tau_m > tau_s else"),
 ("fasta rule2", "else tau_s - 0.5 * tau_m", "else tau_s - tau_m"),
 ("fasta tau_s", "tau_s = float(np.vdot(dx, dx).real) / dxdg", "tau_s = 2.0 * float(np.vdot(dx, dx).real) / dxdg"),
 ("fasta fallback", "else 1.5 * tau", "else 2.0 * tau"),
 ("fasta shrink", "shrink: float = 0.5", "shrink: float = 0.25"),
 ("fasta slack", "bound + 1e-6 * abs(f_max)", "bound + 1e-2 * abs(f_max)"),
 ("fasta no slack", "bound + 1e-6 * abs(f_max)", "bound"),
 ("fasta tau0", "    tau = 1.0 / lipschitz(optics)\n    x = (", "    tau = 2.0 / lipschitz(optics)\n    x = ("),
 ("fasta maxbt", "max_backtracks: int = 20", "max_backtracks: int = 3"),
 ("detect ge", "return m2 > thr2", "return m2 >= thr2"),
 ("detect rel not squared", "thr2 = np.float32(rel * rel) * np.float32(m2.max())", "thr2 = np.float32(rel) * np.float32(m2.max())"),
 ("detect 6-conn", "structure=np.ones((3, 3, 3), dtype=bool)", "structure=None"),
 ("detect minvox", "if count[c] <= min_vox:", "if count[c] < min_vox:"),
 ("detect weight sq", "w = np.abs(np.asarray(x, dtype=np.complex128))", "w = np.abs(np.asarray(x, dtype=np.complex128)) ** 2"),
 ("detect centroid swap", "centroid=(sx[c] / sw[c], sy[c] / sw[c], sz[c] / sw[c])", "centroid=(sy[c] / sw[c], sx[c] / sw[c], sz[c] / sw[c])"),
 ("detect f64 decision", "    xr = np.ascontiguousarray(x.real, dtype=np.float32)\n    xi = np.ascontiguousarray(x.imag, dtype=np.float32)", "    xr = np.ascontiguousarray(x.real, dtype=np.float64)\n    xi = np.ascontiguousarray(x.imag, dtype=np.float64)"),
 ("coo col-major", "j, i = np.nonzero(nzmask)          # row-major order", "i, j = np.nonzero(nzmask.T)"),
 ("coo nz real only", "nzmask = (plane.real != 0) | (plane.imag != 0)", "nzmask = (plane.real != 0)"),
 ("coo expand swap", "x[k, rows[a:b], cols[a:b]] = vals[a:b]", "x[k, cols[a:b], rows[a:b]] = vals[a:b]"),
 ("coo bytes", "return 24 * nnz", "return 16 * nnz"),
 ("freq pitch", "fx = np.fft.fftfreq(optics.nx, d=optics.pitch)", "fx = np.fft.fftfreq(optics.nx, d=2 * optics.pitch)"),
 ("evanescent keep", "return np.where(propagating, np.exp(2j * np.pi * z * kappa), 0.0)", "return np.exp(2j * np.pi * z * kappa)"),
 ("meshgrid swap", 'return np.meshgrid(fy, fx, indexing="ij")', 'return np.meshgrid(fx, fy, indexing="ij")[::-1]'),
 ("data term real part", "return float(np.vdot(r, r).real)", "return float(np.sum(r.real ** 2))"),
 ("detect first last", "np.minimum.at(first, lab, idx)", "np.maximum.at(first, lab, idx)"),
 ("coo offsets", "offsets[k + 1] = offsets[k] + len(j)", "offsets[k + 1] = len(j)"),
 ("proj radius", "scale = 1.0 / np.maximum(1.0, norm)", "scale = 1.0 / np.maximum(0.5, norm)"),
 ("soft real modulus", "    mag = np.abs(u)\n    with", "    mag = np.abs(u.real)\n    with"),
 ("tv_norm dims", "dx, dy, dzz = grad_op(x, dims)\n    return float", "dx, dy, dzz = grad_op(x, 3)\n    return float"),
 ("fgp keep p_prev", "        p_prev, t = p, t_next", "        t = t_next"),
 ("fasta grad at old", "g_new = grad_data(x_new, b, optics)", "g_new = grad_data(x, b, optics)"),
 ("fasta hist old f", "f_hist.append(f_new)", "f_hist.append(f_hist[-1])"),
 ("fista ista keeps y", "            t_next = 1.0\n            y_next = x.copy()\n        x_prev", "            t_next = 1.0\n            y_next = y\n        x_prev"),
 ("adjoint spectrum once", "out[j] = np.fft.ifft2(np.conj(transfer_function(optics, z)) * spectrum)", "out[j] = np.fft.ifft2(np.conj(transfer_function(optics, z)) * spectrum) / optics.nz"),
 ("forward skips last plane", "    for j, z in enumerate(optics.depths()):\n        out += propagate", "    for j, z in enumerate(optics.depths()[:-1]):\n        out += propagate"),
 ("detect centroid z", "sz = np.bincount(lab, weights=wv * kz, minlength=n)", "sz = np.bincount(lab, weights=wv * jy, minlength=n)"),
]

UNET = [
 ("relu abs", "return np.maximum(np.asarray(x, np.float64), 0.0)", "return np.abs(np.asarray(x, np.float64))"),
 ("up scale", "def upsample2(x):\n    \"\"\"Nearest-neighbour 2x upsampling.\"\"\"\n    return np.repeat(", "def upsample2(x):\n    \"\"\"Nearest-neighbour 2x upsampling.\"\"\"\n    return 2 * np.repeat("),
 ("upgrad scale", "return np.asarray(gy, np.float64).reshape(d // 2, 2, h // 2, 2, w // 2, 2, c).sum(axis=(1, 3, 5))", "return 2 * np.asarray(gy, np.float64).reshape(d // 2, 2, h // 2, 2, w // 2, 2, c).sum(axis=(1, 3, 5))"),
 ("pool max", ".mean(axis=(1, 3, 5))", ".max(axis=(1, 3, 5))"),
 ("poolgrad 4", "2, 2) / 8.0", "2, 2) / 4.0"),
 ("dgrad shift sign", "gx += _shift(gy, -dz, -dy, -dx) @ w[:, t, :]", "gx += _shift(gy, dz, dy, dx) @ w[:, t, :]"),
 ("wgrad transpose", "gw[:, t, :] = g2.T @ _shift(x, dz, dy, dx).reshape(-1, cin)", "gw[:, t, :] = g2.T @ _shift(x, -dz, -dy, -dx).reshape(-1, cin)"),
 ("conv bias twice", "        y += np.asarray(b, np.float64)", "        y += 2 * np.asarray(b, np.float64)"),
 ("offsets order", "OFFSETS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]", "OFFSETS = [(dz, dy, dx) for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1)]"),
]

MUTANTS = ([("rihv_oracle.py", CORE_TESTS) + m for m in CORE]
           + [("unet_oracle.py", UNET_TESTS) + m for m in UNET])


def run(mutant):
    fname, tests, name, old, new = mutant
    text = open(os.path.join(ROOT, "oracle", fname)).read()
    if text.count(old) != 1:
        return name, "pattern not found once (the oracle changed: update the mutant)"
    d = tempfile.mkdtemp(prefix="oracle_mutant_")
    try:
        for sub in ("oracle", "tests", "paper_1904_04884_gb300"):
            shutil.copytree(os.path.join(ROOT, sub), os.path.join(d, sub),
                            ignore=shutil.ignore_patterns("lib", "_build", "__pycache__", "*.so",
                                                          "csrc"))
        with open(os.path.join(d, "oracle", fname), "w") as f:
            f.write(text.replace(old, new))
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                            "-m", "not gpu"] + tests, cwd=d, capture_output=True, text=True)
    finally:
        shutil.rmtree(d, ignore_errors=True)
    return name, "killed" if r.returncode != 0 else "SURVIVED"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("-j", type=int, default=os.cpu_count() or 1)
    ap.add_argument("names", nargs="*")
    a = ap.parse_args()
    sel = [m for m in MUTANTS if not a.names or any(s in m[2] for s in a.names)]
    unexpected = 0
    with ThreadPoolExecutor(a.j) as ex:
        for name, res in ex.map(run, sel):
            note = " (equivalent mutant)" if name in EQUIVALENT else ""
            print(f"{name:28s} {res}{note}", flush=True)
            unexpected += (res != "killed") and name not in EQUIVALENT
    print(f"{len(sel)} mutants, {unexpected} unexpected survivors")
    return 1 if unexpected else 0


if __name__ == "__main__":
    sys.exit(main())
