"""Python binding of librihv (ctypes; argument marshalling only).

Every computation runs in the CUDA library; this module converts tensors and
arrays to raw pointers, checks shapes and dtypes, and raises ``RihvError`` on a
non-zero status. Importing works without a GPU; the first call that needs the
library raises if ``lib/librihv.so`` has not been built.

Accepted buffers: torch tensors (CUDA for device arguments, CPU for host
arguments), numpy arrays (host), or raw integer addresses.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "librihv.so")

STATUS = {0: "RIHV_OK", 1: "RIHV_ERR_INVALID_ARG", 2: "RIHV_ERR_CUDA", 3: "RIHV_ERR_OOM",
          4: "RIHV_ERR_NONFINITE", 5: "RIHV_ERR_TIMEOUT", 6: "RIHV_ERR_UNSUPPORTED_SIZE"}

EXPORTS = ["rihv_default_options", "rihv_create", "rihv_destroy", "rihv_set_stream",
           "rihv_set_options", "rihv_forward", "rihv_adjoint", "rihv_prox_fused_lasso",
           "rihv_solve", "rihv_detect", "rihv_detect_coo", "rihv_fasta_steps", "rihv_set_profiling", "rihv_stage_times",
           "rihv_step_size", "rihv_last_error", "rihv_batch_create", "rihv_batch_solve",
           "rihv_batch_destroy", "rihv_autotune", "rihv_tv_schedule", "rihv_tv_split_plan"]

STAGES = ["forward", "adjoint", "tv", "finalize", "objective", "detect", "setup",
          "tv_first", "tv_mid", "tv_final"]


def _particles(arr, n, max_out):
    out = []
    for k in range(min(n, max_out)):
        p = arr[k]
        out.append(dict(centroid=(p.cx, p.cy, p.cz), nvox=p.nvox, weight=p.weight,
                        first=p.first))
    return out


class RihvError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("tv_dims", ctypes.c_int), ("restart", ctypes.c_int),
                ("accelerate", ctypes.c_int), ("n_inner", ctypes.c_int),
                ("check_every", ctypes.c_int), ("tol", ctypes.c_double),
                ("f_star", ctypes.c_double), ("tv_steps_per_launch", ctypes.c_int),
                ("fuse_finalize", ctypes.c_int), ("skip_empty_planes", ctypes.c_int),
                ("tv_zchunk", ctypes.c_int), ("fft_rows_per_cta", ctypes.c_int),
                ("tv_fgp", ctypes.c_int), ("solver", ctypes.c_int), ("tv_split", ctypes.c_int)]


class Particle(ctypes.Structure):
    _fields_ = [("cx", ctypes.c_double), ("cy", ctypes.c_double), ("cz", ctypes.c_double),
                ("weight", ctypes.c_double), ("first", ctypes.c_int64), ("nvox", ctypes.c_int32),
                ("pad_", ctypes.c_int32)]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads librihv.so and declares its signatures. Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"librihv.so not found at {path}; build it with "
                           "`python -m paper_1904_04884_gb300.build`")
    L = ctypes.CDLL(path)
    vp, i, d, f = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_float
    H = ctypes.c_void_p
    sig = {
        "rihv_default_options": (None, [ctypes.POINTER(Options)]),
        "rihv_create": (i, [i, i, i, d, d, d, d, ctypes.POINTER(H)]),
        "rihv_destroy": (i, [H]),
        "rihv_set_stream": (i, [H, vp]),
        "rihv_set_options": (i, [H, ctypes.POINTER(Options)]),
        "rihv_forward": (i, [H, vp, vp]),
        "rihv_adjoint": (i, [H, vp, vp]),
        "rihv_prox_fused_lasso": (i, [H, vp, f, f, i, vp]),
        "rihv_solve": (i, [H, vp, f, f, i, vp, vp, vp, ctypes.POINTER(i)]),
        "rihv_detect": (i, [H, vp, f, i, ctypes.POINTER(Particle), i, ctypes.POINTER(i)]),
        "rihv_detect_coo": (i, [H, vp, vp, vp, vp, ctypes.c_longlong, f, i,
                                ctypes.POINTER(Particle), i, ctypes.POINTER(i)]),
        "rihv_fasta_steps": (i, [H, ctypes.POINTER(d), i, ctypes.POINTER(i), ctypes.POINTER(i)]),
        "rihv_set_profiling": (i, [H, i]),
        "rihv_stage_times": (i, [H, ctypes.POINTER(d), ctypes.POINTER(ctypes.c_longlong), i]),
        "rihv_step_size": (i, [H, ctypes.POINTER(d)]),
        "rihv_last_error": (ctypes.c_char_p, [H]),
        "rihv_batch_create": (i, [ctypes.POINTER(H), i, ctypes.POINTER(H)]),
        "rihv_batch_solve": (i, [H, ctypes.POINTER(vp), f, f, i, ctypes.POINTER(vp),
                                 ctypes.POINTER(vp), ctypes.POINTER(vp)]),
        "rihv_batch_destroy": (i, [H]),
        "rihv_batch_iterations": (i, [H, ctypes.POINTER(i)]),
        "rihv_autotune": (i, [H, ctypes.c_char_p, ctypes.POINTER(i)]),
        "rihv_tv_schedule": (i, [H, i, ctypes.POINTER(i)]),
        "rihv_tv_split_plan": (i, [i, i, i, i, i, i, ctypes.POINTER(i)]),
        "rihv_coo_compact": (i, [H, vp, vp, vp, vp, vp, ctypes.c_longlong,
                                 ctypes.POINTER(ctypes.c_longlong)]),
        "rihv_coo_expand": (i, [H, vp, vp, vp, vp, ctypes.c_longlong, vp]),
        "rihv_selftest_bounded_wait": (i, [H, i]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _ptr(buf, *, device=None, dtype=None, numel=None, name="buffer"):
    """Raw address of a torch tensor, numpy array or int (None -> 0)."""
    if buf is None:
        return None
    if isinstance(buf, int):
        return buf
    if isinstance(buf, np.ndarray):
        if device is True:
            raise ValueError(f"{name} must be device memory")
        if not buf.flags.c_contiguous:
            raise ValueError(f"{name} must be C-contiguous")
        if dtype is not None and buf.dtype != np.dtype(dtype):
            raise ValueError(f"{name} must be {np.dtype(dtype)}, got {buf.dtype}")
        if numel is not None and buf.size != numel:
            raise ValueError(f"{name} has {buf.size} elements, expected {numel}")
        return buf.ctypes.data
    # torch tensor
    if not buf.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if device is True and not buf.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None:
        want = {"complex64": "torch.complex64", "float32": "torch.float32",
                "float64": "torch.float64", "int32": "torch.int32",
                "int64": "torch.int64"}[np.dtype(dtype).name]
        if str(buf.dtype) != want:
            raise ValueError(f"{name} must be {want}, got {buf.dtype}")
    if numel is not None and buf.numel() != numel:
        raise ValueError(f"{name} has {buf.numel()} elements, expected {numel}")
    return buf.data_ptr()


class Rihv:
    """One reconstruction grid and optics (a ``rihv_handle``)."""

    def __init__(self, nx, ny, nz, wavelength, pitch, z0, dz, stream=None):
        self.L = load_library()
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.nxy = self.nx * self.ny
        self.nvox = self.nxy * self.nz
        h = ctypes.c_void_p()
        self._check(self.L.rihv_create(self.nx, self.ny, self.nz, float(wavelength), float(pitch),
                                       float(z0), float(dz), ctypes.byref(h)), None)
        self.h = h
        if stream is not None:
            self.set_stream(stream)

    # -- plumbing ---------------------------------------------------------
    def _check(self, st, h):
        if st != 0:
            msg = self.L.rihv_last_error(h)
            raise RihvError(st, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "h", None):
            self.L.rihv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t address, or None."""
        ptr = getattr(stream, "cuda_stream", stream)
        self._check(self.L.rihv_set_stream(self.h, ptr), self.h)

    def set_options(self, **kw):
        o = Options()
        self.L.rihv_default_options(ctypes.byref(o))
        for k, v in kw.items():
            if not hasattr(o, k):
                raise KeyError(k)
            setattr(o, k, v)
        self._check(self.L.rihv_set_options(self.h, ctypes.byref(o)), self.h)
        self.options = o

    def step_size(self) -> float:
        t = ctypes.c_double()
        self._check(self.L.rihv_step_size(self.h, ctypes.byref(t)), self.h)
        return t.value

    # -- operators ----------------------------------------------------------
    def rihv_forward(self, x, out):
        self._check(self.L.rihv_forward(
            self.h, _ptr(x, device=True, dtype="complex64", numel=self.nvox, name="x"),
            _ptr(out, device=True, dtype="complex64", numel=self.nxy, name="out")), self.h)

    def rihv_adjoint(self, r, out):
        self._check(self.L.rihv_adjoint(
            self.h, _ptr(r, device=True, dtype="complex64", numel=self.nxy, name="r"),
            _ptr(out, device=True, dtype="complex64", numel=self.nvox, name="out")), self.h)

    def rihv_prox_fused_lasso(self, v, t_l1, t_tv, inner_iters, x_out):
        self._check(self.L.rihv_prox_fused_lasso(
            self.h, _ptr(v, device=True, dtype="complex64", numel=self.nvox, name="v"),
            float(t_l1), float(t_tv), int(inner_iters),
            _ptr(x_out, device=True, dtype="complex64", numel=self.nvox, name="x_out")), self.h)

    def rihv_solve(self, hologram, lambda_l1, lambda_tv, iters, x_out, x0=None, trace=None):
        """Runs FISTA; returns the number of iterations run."""
        done = ctypes.c_int()
        self._check(self.L.rihv_solve(
            self.h, _ptr(hologram, dtype="float32", numel=self.nxy, name="hologram"),
            float(lambda_l1), float(lambda_tv), int(iters),
            _ptr(x0, dtype="complex64", numel=self.nvox, name="x0"),
            _ptr(x_out, dtype="complex64", numel=self.nvox, name="x_out"),
            _ptr(trace, dtype="float64", name="trace"), ctypes.byref(done)), self.h)
        return done.value

    def rihv_detect(self, x, rel_thresh=2.0 / 256.0, min_vox=5, max_out=1 << 20):
        """Returns a list of particle dicts ordered by smallest voxel index.
        x = None detects on the result of the last solve on this handle."""
        n = ctypes.c_int()
        arr = (Particle * max(1, max_out))()
        self._check(self.L.rihv_detect(
            self.h, _ptr(x, device=True, dtype="complex64", numel=self.nvox, name="x") or None,
            float(rel_thresh), int(min_vox), arr, int(max_out), ctypes.byref(n)), self.h)
        return _particles(arr, n.value, max_out)

    def rihv_detect_coo(self, offsets, rows, cols, vals, rel_thresh=2.0 / 256.0, min_vox=5,
                        max_out=1 << 20):
        """Detection on a per-plane COO form (as rihv_coo_compact returns it);
        the same particles as rihv_detect on the expanded volume."""
        n = ctypes.c_int()
        nnz = int(rows.numel())
        arr = (Particle * max(1, max_out))()
        self._check(self.L.rihv_detect_coo(
            self.h, _ptr(offsets, device=True, dtype="int64", numel=self.nz + 1, name="offsets"),
            _ptr(rows, device=True, dtype="int32", name="rows") if nnz else None,
            _ptr(cols, device=True, dtype="int32", name="cols") if nnz else None,
            _ptr(vals, device=True, dtype="complex64", name="vals") if nnz else None, nnz,
            float(rel_thresh), int(min_vox), arr, int(max_out), ctypes.byref(n)), self.h)
        return _particles(arr, n.value, max_out)

    def rihv_coo_compact(self, x=None):
        """Per-plane COO form of x (None: the last solve's result) as device
        tensors (plane_offsets int64 [nz+1], rows int32, cols int32, vals
        complex64); plane k's entries lie at [offsets[k], offsets[k+1]) in
        row-major order."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device()) if x is None else x.device
        off = torch.empty(self.nz + 1, dtype=torch.int64, device=dev)
        xp = _ptr(x, device=True, dtype="complex64", numel=self.nvox, name="x") or None
        nnz = ctypes.c_longlong()
        st = self.L.rihv_coo_compact(self.h, xp, off.data_ptr(), None, None, None, 0,
                                     ctypes.byref(nnz))
        n = nnz.value
        if st != 0 and n == 0:
            self._check(st, self.h)
        rows = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        cols = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
        vals = torch.empty(max(n, 1), dtype=torch.complex64, device=dev)
        if n > 0:
            self._check(self.L.rihv_coo_compact(self.h, xp, off.data_ptr(), rows.data_ptr(),
                                                cols.data_ptr(), vals.data_ptr(), n,
                                                ctypes.byref(nnz)), self.h)
        return off, rows[:n], cols[:n], vals[:n]

    def rihv_coo_expand(self, offsets, rows, cols, vals, x_out):
        """Dense volume x_out from a per-plane COO form (zeros elsewhere)."""
        n = int(rows.numel())
        self._check(self.L.rihv_coo_expand(
            self.h, _ptr(offsets, device=True, dtype="int64", numel=self.nz + 1, name="offsets"),
            _ptr(rows, device=True, dtype="int32", name="rows") if n else None,
            _ptr(cols, device=True, dtype="int32", name="cols") if n else None,
            _ptr(vals, device=True, dtype="complex64", name="vals") if n else None, n,
            _ptr(x_out, device=True, dtype="complex64", numel=self.nvox, name="x_out")), self.h)

    def rihv_fasta_steps(self):
        """(accepted step sizes, backtracking halvings) of the last FASTA solve."""
        n, bt = ctypes.c_int(), ctypes.c_int()
        self._check(self.L.rihv_fasta_steps(self.h, None, 0, ctypes.byref(n), ctypes.byref(bt)),
                    self.h)
        arr = (ctypes.c_double * max(1, n.value))()
        self._check(self.L.rihv_fasta_steps(self.h, arr, n.value, ctypes.byref(n),
                                            ctypes.byref(bt)), self.h)
        return list(arr[:n.value]), bt.value

    fasta_steps = rihv_fasta_steps
    detect_coo = rihv_detect_coo
    coo_compact = rihv_coo_compact
    coo_expand = rihv_coo_expand

    def rihv_autotune(self, cache_path=None):
        """Times the TV z-chunk / steps per launch, the column-pass z-groups and
        the row-pass FFT tile (rows per CTA) on this handle and applies the
        fastest; returns (z_chunk, steps_per_launch, planes_per_group,
        rows_per_cta). With cache_path the result is looked up / stored."""
        out = (ctypes.c_int * 4)()
        path = cache_path.encode() if cache_path else None
        self._check(self.L.rihv_autotune(self.h, path, out), self.h)
        return tuple(out)

    autotune = rihv_autotune

    def rihv_tv_schedule(self, final=False):
        """(planes per z-chunk, split tile, planes per z-chunk from the split
        tile on, 0 without a split) of the two-step TV launches of a solve:
        final=False for the launches reading the dual, True for the fused
        finalize."""
        out = (ctypes.c_int * 3)()
        self._check(self.L.rihv_tv_schedule(self.h, int(bool(final)), out), self.h)
        return tuple(out)

    tv_schedule = rihv_tv_schedule

    # -- profiling ----------------------------------------------------------
    def rihv_selftest_bounded_wait(self, polls=4096):
        """Runs the library's bounded mbarrier wait on a barrier nothing
        arrives on; returns the status code without raising (5,
        RIHV_ERR_TIMEOUT, is the expected outcome)."""
        return self.L.rihv_selftest_bounded_wait(self.h, int(polls))

    def set_profiling(self, on):
        """False/0 off; True/1 stage events; 2 also events around every TV launch."""
        self._check(self.L.rihv_set_profiling(self.h, int(on)), self.h)

    def stage_times(self):
        """{stage: (ms, launches)} accumulated since the last call."""
        n = len(STAGES)
        ms = (ctypes.c_double * n)()
        nl = (ctypes.c_longlong * n)()
        self._check(self.L.rihv_stage_times(self.h, ms, nl, n), self.h)
        return {s: (ms[i], nl[i]) for i, s in enumerate(STAGES)}

    # short aliases
    forward = rihv_forward
    adjoint = rihv_adjoint
    prox_fused_lasso = rihv_prox_fused_lasso
    solve = rihv_solve
    detect = rihv_detect


class Batch:
    """Handles solved together as one CUDA graph (rihv_batch_*)."""

    def __init__(self, handles):
        self.L = load_library()
        self.handles = list(handles)
        arr = (ctypes.c_void_p * len(self.handles))(*[h.h.value for h in self.handles])
        b = ctypes.c_void_p()
        st = self.L.rihv_batch_create(arr, len(self.handles), ctypes.byref(b))
        if st != 0:
            raise RihvError(st, self.L.rihv_last_error(None).decode())
        self.b = b

    def solve(self, holograms, lambda_l1, lambda_tv, iters, x_outs, x0s=None, traces=None):
        n = len(self.handles)
        vp = ctypes.c_void_p
        holo = (vp * n)(*[_ptr(g, dtype="float32", numel=h.nxy, name="hologram")
                          for g, h in zip(holograms, self.handles)])
        outs = (vp * n)(*[_ptr(x, dtype="complex64", numel=h.nvox, name="x_out")
                          for x, h in zip(x_outs, self.handles)])
        x0 = None if x0s is None else (vp * n)(*[_ptr(x, dtype="complex64", numel=h.nvox,
                                                      name="x0")
                                                 for x, h in zip(x0s, self.handles)])
        tr = None if traces is None else (vp * n)(*[_ptr(t, dtype="float64", name="trace")
                                                    for t in traces])
        st = self.L.rihv_batch_solve(self.b, holo, float(lambda_l1), float(lambda_tv), int(iters),
                                     x0, outs, tr)
        if st != 0:
            msgs = [self.L.rihv_last_error(h.h).decode() for h in self.handles]
            raise RihvError(st, "; ".join(m for m in msgs if m))

    def iterations(self):
        """Iterations each handle ran in the last solve (handles with a stop
        test, f_star > 0, stop at their first check that meets it)."""
        out = (ctypes.c_int * len(self.handles))()
        st = self.L.rihv_batch_iterations(self.b, out)
        if st != 0:
            raise RihvError(st, "rihv_batch_iterations failed")
        return list(out)

    def close(self):
        if getattr(self, "b", None):
            self.L.rihv_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rihv_tv_split_plan(nx, ny, nz, final, zchunk, sms=152):
    """(split tile, planes per z-chunk from it on) that the library's split
    rule gives a two-step TV launch of an nx x ny x nz volume with z-chunks of
    `zchunk` planes on `sms` SMs; (0, 0) keeps equal chunks. Host only."""
    L = load_library()
    out = (ctypes.c_int * 2)()
    st = L.rihv_tv_split_plan(int(nx), int(ny), int(nz), int(final), int(zchunk), int(sms), out)
    if st != 0:
        msg = L.rihv_last_error(None)
        raise RihvError(st, msg.decode() if msg else "rihv_tv_split_plan failed")
    return tuple(out)


def rihv_prox_fused_lasso_noalloc(v, x_out, nz, ny, nx, tv_dims, t_l1, t_tv, inner_iters,
                                  stream=None):
    """The fused-lasso prox without any device allocation (static scratch in the
    library; see include/rihv.h). For callers that cannot allocate: hosts
    whose device memory is a fixed arena of their own, and services that stop
    allocating after start-up. Volumes up to 1,048,576 voxels; nx must be
    even; v, x_out and the stream on the current device. Calls that overlap
    on the GPU share the scratch and race. A TV wait that gave up leaves x_out
    all NaN."""
    L = load_library()
    fn = L.rihv_prox_fused_lasso_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                   ctypes.c_int, ctypes.c_float, ctypes.c_float, ctypes.c_int, ctypes.c_void_p]
    n = int(nx) * int(ny) * int(nz)
    st = fn(_ptr(v, device=True, dtype="complex64", numel=n, name="v"),
            _ptr(x_out, device=True, dtype="complex64", numel=n, name="x_out"),
            int(nx), int(ny), int(nz), int(tv_dims), float(t_l1), float(t_tv), int(inner_iters),
            getattr(stream, "cuda_stream", stream))
    if st != 0:
        msg = L.rihv_last_error(None)
        raise RihvError(st, msg.decode() if msg else "rihv_prox_fused_lasso_noalloc failed")
