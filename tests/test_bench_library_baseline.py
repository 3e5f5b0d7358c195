"""bench.py's library baseline (the FISTA iteration with PyTorch operators,
as the paper describes its own GPU code) against the FP64 oracle, run with
PyTorch on the CPU at the 64 x 64 x 16 size: the operators and the prox to
the per-operator tolerance, five FISTA iterations to the solve tolerance."""
import importlib.util
import os

import numpy as np
import torch

from oracle import rihv_oracle as O
from paper_1904_04884_gb300 import synth, workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_lib_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _rel(a, b):
    a = np.asarray(a, np.complex128)
    b = np.asarray(b, np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex64))


def test_library_baseline_matches_the_oracle():
    w = workloads.TINY
    op = O.Optics(*w.optics_tuple())
    lf = _bench().LibraryFista(w, torch.device("cpu"))
    assert abs(lf.tau - 1.0 / O.lipschitz(op)) <= 1e-7 * lf.tau
    x = synth.random_complex(synth.Stream(3), op.shape)
    assert _rel(lf.forward(_t(x)).numpy(), O.forward(x, op)) <= 1e-5
    r = synth.random_complex(synth.Stream(4), (op.ny, op.nx))
    assert _rel(lf.adjoint(_t(r)).numpy(), O.adjoint(r, op)) <= 1e-5
    for dims in (3, 2):
        got = lf.soft(lf.tv_prox(_t(x), 0.3, 7, dims), 0.2).numpy()
        assert _rel(got, O.prox_fused_lasso(x, 0.2, 0.3, 7, dims)) <= 1e-5
    a = w.opacity().astype(np.float64)
    b = synth.intensity_hologram(O.forward(a, op), w.sigma, w.noise())
    got = lf.solve(_t(b), w.lam_l1, w.lam_tv, 5, w.n_inner, 3).numpy()
    ref, _ = O.fista(b.astype(np.float64), op, w.lam_l1, w.lam_tv, 5, w.n_inner)
    assert _rel(got, ref) <= 1e-3
