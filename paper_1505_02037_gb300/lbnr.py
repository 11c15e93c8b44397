"""Thin Python binding of the lbnr C-ABI (include/lbnr.h).

Every function here only marshals arguments: the lattice Boltzmann step,
the moments and the constraint reductions all run in liblbnr.so's CUDA
kernels. PyTorch provides the device memory (one uint8 tensor handed to the
library as its workspace) and the CUDA stream. There is no CPU fallback: if
the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

LBNR_D1Q3, LBNR_D2Q9, LBNR_D3Q19 = 1, 2, 3
LBNR_F64, LBNR_F32, LBNR_DEV_F32, LBNR_DEV_BF16, LBNR_DEV_F16 = 0, 1, 2, 3, 4
LBNR_GEODESIC, LBNR_HARMONIC, LBNR_ONE_PLUS_LOG = 0, 1, 2
LBNR_STREAM_AUTO, LBNR_STREAM_PINGPONG, LBNR_STREAM_AA = 0, 1, 2
LBNR_DERIV_SYNC, LBNR_DERIV_LAG = 0, 1
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ENONFINITE", -5: "ETIMEOUT",
          -6: "ESTATE"}
Q_OF = {1: 3, 2: 9, 3: 19}
STORAGE_NAMES = {"f64": 0, "f32": 1, "dev_f32": 2, "dev_bf16": 3, "dev_f16": 4}


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64)]


class Opts(ctypes.Structure):
    _fields_ = [("slicing", ctypes.c_int32), ("storage", ctypes.c_int32),
                ("streaming", ctypes.c_int32), ("sources_on", ctypes.c_int32),
                ("cuda_stream", ctypes.c_void_p), ("dev_buffer", ctypes.c_void_p),
                ("dev_bytes", ctypes.c_uint64), ("deriv_mode", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class RunDesc(ctypes.Structure):
    _fields_ = [("vset", ctypes.c_int32), ("slicing", ctypes.c_int32), ("grid", Grid),
                ("tau", ctypes.c_double), ("dx", ctypes.c_double), ("steps", ctypes.c_int64)]


class BatchOpts(ctypes.Structure):
    _fields_ = [("storage", ctypes.c_int32), ("block", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("sources_on", ctypes.c_int32),
                ("cuda_stream", ctypes.c_void_p), ("wait_limit_ns", ctypes.c_int64),
                ("test_drop_arrival_run", ctypes.c_int32), ("replan", ctypes.c_int32),
                ("deriv_mode", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class LbnrError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lbnr error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


class NonFiniteError(LbnrError):
    pass


_lib = None


def library(path: str | None = None):
    """Loads liblbnr.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or os.environ.get("LBNR_LIB") or _build.build()
    L = ctypes.CDLL(path)
    vp, i64, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
    L.lbnr_default_opts.argtypes = [ctypes.POINTER(Opts)]
    L.lbnr_default_opts.restype = None
    L.lbnr_workspace_bytes.argtypes = [ctypes.POINTER(Grid), ctypes.c_int, ctypes.POINTER(Opts),
                                       ctypes.POINTER(ctypes.c_uint64)]
    L.lbnr_create.argtypes = [ctypes.POINTER(Grid), ctypes.c_int, ctypes.c_double,
                              ctypes.c_double, ctypes.c_double, ctypes.POINTER(Opts),
                              ctypes.POINTER(vp)]
    for name in ("lbnr_init", "lbnr_moments", "lbnr_constraints", "lbnr_get_distributions",
                 "lbnr_set_distributions"):
        getattr(L, name).argtypes = [vp, dp]
    L.lbnr_get_cells.argtypes = [vp, i64, ctypes.POINTER(ctypes.c_int64), dp]
    L.lbnr_step.argtypes = [vp, i64]
    L.lbnr_step_timed.argtypes = [vp, i64, dp]
    L.lbnr_status.argtypes = [vp]
    L.lbnr_get_lagged.argtypes = [vp, dp]
    L.lbnr_set_lagged.argtypes = [vp, dp]
    L.lbnr_deriv_mode.argtypes = [vp]
    L.lbnr_steps_done.argtypes = [vp]
    L.lbnr_steps_done.restype = i64
    L.lbnr_q.argtypes = [vp]
    L.lbnr_streaming.argtypes = [vp]
    L.lbnr_num_variants.argtypes = [vp]
    L.lbnr_variant_name.argtypes = [vp, ctypes.c_int]
    L.lbnr_variant_name.restype = ctypes.c_char_p
    L.lbnr_set_variant.argtypes = [vp, ctypes.c_int]
    L.lbnr_set_fluid.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double]
    L.lbnr_set_shift.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double]
    L.lbnr_set_shift_field.argtypes = [vp, vp]
    L.lbnr_fp64_fma_rate.argtypes = [vp, dp]
    L.lbnr_constraint_norms_noalloc.argtypes = [ctypes.c_int, ctypes.POINTER(Grid),
                                                 ctypes.c_double, vp, vp, vp]
    L.lbnr_default_batch_opts.argtypes = [ctypes.POINTER(BatchOpts)]
    L.lbnr_default_batch_opts.restype = None
    L.lbnr_batch_create.argtypes = [ctypes.c_int, ctypes.POINTER(RunDesc),
                                    ctypes.POINTER(BatchOpts), ctypes.POINTER(vp)]
    L.lbnr_batch_configure.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    L.lbnr_batch_init.argtypes = [vp, ctypes.c_int, dp]
    L.lbnr_batch_run.argtypes = [vp, i64]
    L.lbnr_batch_replan.argtypes = [vp]
    L.lbnr_batch_status.argtypes = [vp, ctypes.POINTER(ctypes.c_int32)]
    L.lbnr_batch_get_distributions.argtypes = [vp, ctypes.c_int, dp]
    i32p = ctypes.POINTER(ctypes.c_int32)
    L.lbnr_batch_plan.argtypes = [vp, i32p, i32p, i32p, i32p]
    L.lbnr_batch_steps_done.argtypes = [vp, ctypes.c_int]
    L.lbnr_batch_steps_done.restype = i64
    L.lbnr_batch_destroy.argtypes = [vp]
    L.lbnr_batch_destroy.restype = None
    L.lbnr_batch_last_error.argtypes = [vp]
    L.lbnr_batch_last_error.restype = ctypes.c_char_p
    L.lbnr_destroy.argtypes = [vp]
    L.lbnr_destroy.restype = None
    L.lbnr_last_error.argtypes = [vp]
    L.lbnr_last_error.restype = ctypes.c_char_p
    L.lbnr_ad_create.argtypes = [ctypes.POINTER(Grid), ctypes.c_int, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                 vp, ctypes.POINTER(vp)]
    L.lbnr_ad_init.argtypes = [vp, dp, ctypes.c_int]
    L.lbnr_ad_step.argtypes = [vp, i64]
    L.lbnr_ad_step_timed.argtypes = [vp, i64, dp]
    for name in ("lbnr_ad_moments", "lbnr_ad_get_distributions", "lbnr_ad_set_distributions"):
        getattr(L, name).argtypes = [vp, dp]
    L.lbnr_ad_status.argtypes = [vp]
    L.lbnr_ad_set_form.argtypes = [vp, ctypes.c_int]
    L.lbnr_ad_form_blocks.argtypes = [ctypes.c_int]
    L.lbnr_ad_steps_done.argtypes = [vp]
    L.lbnr_ad_steps_done.restype = i64
    L.lbnr_ad_destroy.argtypes = [vp]
    L.lbnr_ad_destroy.restype = None
    L.lbnr_ad_last_error.argtypes = [vp]
    L.lbnr_ad_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(rc, ctx=None, batch=None, ad=None):
    if rc == 0:
        return
    if ad is not None:
        msg = library().lbnr_ad_last_error(ad).decode(errors="replace")
    elif batch is not None:
        msg = library().lbnr_batch_last_error(batch).decode(errors="replace")
    else:
        msg = library().lbnr_last_error(ctx).decode(errors="replace")
    if rc == -4:
        raise NonFiniteError(rc, msg)
    raise LbnrError(rc, msg)


def _dptr(a: np.ndarray):
    if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
        raise TypeError("expected a C-contiguous float64 array")
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _host_ptr(a):
    """Pointer of a host float64 buffer: numpy array or (pinned) CPU tensor."""
    if isinstance(a, np.ndarray):
        return _dptr(a)
    import torch
    if isinstance(a, torch.Tensor):
        if a.device.type != "cpu" or a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("expected a contiguous float64 CPU tensor")
        return ctypes.cast(ctypes.c_void_p(a.data_ptr()), ctypes.POINTER(ctypes.c_double))
    raise TypeError(type(a))


# ---------------------------------------------------------------------------
# C-ABI, one Python function per entry point
# ---------------------------------------------------------------------------
def lbnr_default_opts() -> Opts:
    o = Opts()
    library().lbnr_default_opts(ctypes.byref(o))
    return o


def lbnr_workspace_bytes(grid: Grid, vset: int, opts: Opts) -> int:
    out = ctypes.c_uint64(0)
    _check(library().lbnr_workspace_bytes(ctypes.byref(grid), vset, ctypes.byref(opts),
                                          ctypes.byref(out)))
    return out.value


def lbnr_create(grid: Grid, vset: int, tau: float, dx: float, dt: float, opts: Opts):
    ctx = ctypes.c_void_p(0)
    _check(library().lbnr_create(ctypes.byref(grid), vset, tau, dx, dt, ctypes.byref(opts),
                                 ctypes.byref(ctx)))
    return ctx


def lbnr_init(ctx, fields):
    _check(library().lbnr_init(ctx, _host_ptr(fields)), ctx)


def lbnr_step(ctx, n: int):
    _check(library().lbnr_step(ctx, int(n)), ctx)


def lbnr_step_timed(ctx, n: int):
    """Runs n steps kernel by kernel; returns (ms in the moment pass,
    ms in the collide-and-stream kernel)."""
    ms = np.zeros(2)
    _check(library().lbnr_step_timed(ctx, int(n), _dptr(ms)), ctx)
    return float(ms[0]), float(ms[1])


def lbnr_moments(ctx, out):
    _check(library().lbnr_moments(ctx, _host_ptr(out)), ctx)


def lbnr_constraints(ctx, out):
    _check(library().lbnr_constraints(ctx, _host_ptr(out)), ctx)


def lbnr_get_distributions(ctx, out):
    _check(library().lbnr_get_distributions(ctx, _host_ptr(out)), ctx)


def lbnr_get_cells(ctx, cells, out):
    idx = np.ascontiguousarray(np.asarray(cells, dtype=np.int64))
    _check(library().lbnr_get_cells(ctx, len(idx), idx.ctypes.data_as(
        ctypes.POINTER(ctypes.c_int64)), _host_ptr(out)), ctx)


def lbnr_set_distributions(ctx, arr):
    _check(library().lbnr_set_distributions(ctx, _host_ptr(arr)), ctx)


def lbnr_status(ctx):
    _check(library().lbnr_status(ctx), ctx)


def lbnr_get_lagged(ctx, out):
    _check(library().lbnr_get_lagged(ctx, _host_ptr(out)), ctx)


def lbnr_set_lagged(ctx, arr):
    _check(library().lbnr_set_lagged(ctx, _host_ptr(arr)), ctx)


def lbnr_steps_done(ctx) -> int:
    return library().lbnr_steps_done(ctx)


def lbnr_num_variants(ctx) -> int:
    return library().lbnr_num_variants(ctx)


def lbnr_variant_name(ctx, v: int) -> str:
    return library().lbnr_variant_name(ctx, v).decode()


def lbnr_set_variant(ctx, v: int):
    _check(library().lbnr_set_variant(ctx, v), ctx)


def lbnr_set_fluid(ctx, rho0: float, w: float, t0: float):
    _check(library().lbnr_set_fluid(ctx, float(rho0), float(w), float(t0)), ctx)


def lbnr_set_shift(ctx, bx: float, by: float, bz: float):
    _check(library().lbnr_set_shift(ctx, float(bx), float(by), float(bz)), ctx)


def lbnr_set_shift_field(ctx, beta):
    """beta: host float64 [3][cells] (C-contiguous) or None to remove."""
    _check(library().lbnr_set_shift_field(ctx, None if beta is None else _host_ptr(beta)), ctx)


def lbnr_constraint_norms_noalloc(vset: int, grid: Grid, dx: float, d_fields, d_out,
                                  stream=None):
    """Constraint norms of device-resident corrected fields without any device
    allocation (see include/lbnr.h). d_fields: CUDA float64 tensor [16, cells];
    d_out: CUDA float64 tensor [6]; stream: torch CUDA stream or None."""
    import torch
    for t, n in ((d_fields, 16 * grid.nx * grid.ny * grid.nz), (d_out, 6)):
        if (not t.is_cuda or str(t.dtype) != "torch.float64" or not t.is_contiguous()
                or t.numel() != n):
            raise TypeError("expected contiguous CUDA float64 tensors of the right size")
    # the kernels run on the current device: both tensors and the stream must
    # be on it
    dev = d_fields.device
    if d_out.device != dev or (stream is not None and stream.device != dev):
        raise ValueError("d_fields, d_out and the stream must be on the same CUDA device")
    st = ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)
    with torch.cuda.device(dev):
        _check(library().lbnr_constraint_norms_noalloc(
            int(vset), ctypes.byref(grid), float(dx), ctypes.c_void_p(d_fields.data_ptr()),
            ctypes.c_void_p(d_out.data_ptr()), st))


def lbnr_fp64_fma_rate(stream=None) -> float:
    """Measured FP64 FMA rate of the current device in TFLOP/s."""
    out = ctypes.c_double(0)
    st = ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)
    _check(library().lbnr_fp64_fma_rate(st, ctypes.byref(out)))
    return out.value


def lbnr_destroy(ctx):
    library().lbnr_destroy(ctx)


def lbnr_default_batch_opts() -> BatchOpts:
    o = BatchOpts()
    library().lbnr_default_batch_opts(ctypes.byref(o))
    return o


def lbnr_batch_create(runs, opts: BatchOpts):
    arr = (RunDesc * len(runs))(*runs)
    b = ctypes.c_void_p(0)
    _check(library().lbnr_batch_create(len(runs), arr, ctypes.byref(opts), ctypes.byref(b)))
    return b


def lbnr_batch_configure(b, block: int, ctas_per_sm: int):
    _check(library().lbnr_batch_configure(b, int(block), int(ctas_per_sm)), batch=b)


def lbnr_batch_init(b, run: int, fields):
    _check(library().lbnr_batch_init(b, int(run), _host_ptr(fields)), batch=b)


def lbnr_batch_run(b, max_steps: int = -1):
    _check(library().lbnr_batch_run(b, int(max_steps)), batch=b)


def lbnr_batch_replan(b):
    _check(library().lbnr_batch_replan(b), batch=b)


def lbnr_batch_status(b, nruns: int):
    """Returns (worst code, per-run codes); raises nothing."""
    per = (ctypes.c_int32 * nruns)()
    rc = library().lbnr_batch_status(b, per)
    return rc, list(per)


def lbnr_batch_get_distributions(b, run: int, out):
    _check(library().lbnr_batch_get_distributions(b, int(run), _host_ptr(out)), batch=b)


def lbnr_batch_plan(b, nruns: int):
    g, blk, gr = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    teams = (ctypes.c_int32 * nruns)()
    _check(library().lbnr_batch_plan(b, ctypes.byref(g), ctypes.byref(blk), ctypes.byref(gr),
                                     teams))
    return {"grid": g.value, "block": blk.value, "graphed": bool(gr.value), "teams": list(teams)}


def lbnr_batch_steps_done(b, run: int) -> int:
    return library().lbnr_batch_steps_done(b, int(run))


def lbnr_batch_destroy(b):
    library().lbnr_batch_destroy(b)


# ---------------------------------------------------------------------------
# Convenience wrapper: one lattice, torch-owned workspace and stream
# ---------------------------------------------------------------------------
class Lattice:
    """One periodic lattice on the current CUDA device.

    vset: 1 D1Q3, 2 D2Q9, 3 D3Q19; shape (nx, ny, nz); tau is tau/dt; dx = dt.
    storage: "f64", "f32", "dev_f32", "dev_bf16", "dev_f16" (or the code).
    """

    def __init__(self, vset, shape, tau, dx, dt=None, slicing=LBNR_HARMONIC, storage="f64",
                 streaming=LBNR_STREAM_AUTO, sources_on=True, stream=None, device=None,
                 deriv_mode=LBNR_DERIV_SYNC):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("lbnr needs a CUDA device; there is no CPU path")
        self.torch = torch
        self.device = torch.device(device or "cuda")
        library()
        self.vset = int(vset)
        self.Q = Q_OF[self.vset]
        self.shape = tuple(int(s) for s in shape)
        self.cells = self.shape[0] * self.shape[1] * self.shape[2]
        self.storage = STORAGE_NAMES.get(storage, storage)
        self.grid = Grid(*self.shape)
        self.stream = stream or torch.cuda.current_stream(self.device)
        if self.stream.cuda_stream == 0:
            # the legacy default stream cannot be graph-captured: use our own
            self.stream = torch.cuda.Stream(self.device)
        o = lbnr_default_opts()
        o.slicing = int(slicing)
        o.storage = int(self.storage)
        o.sources_on = int(bool(sources_on))
        o.deriv_mode = {"sync": LBNR_DERIV_SYNC, "lag": LBNR_DERIV_LAG}.get(deriv_mode, deriv_mode)
        o.cuda_stream = ctypes.c_void_p(self.stream.cuda_stream)
        if streaming == LBNR_STREAM_AUTO:
            o.streaming = LBNR_STREAM_PINGPONG
            need_pp = lbnr_workspace_bytes(self.grid, self.vset, o)
            free, _ = torch.cuda.mem_get_info(self.device)
            streaming = LBNR_STREAM_PINGPONG if need_pp <= 0.9 * free else LBNR_STREAM_AA
        o.streaming = int(streaming)
        nbytes = lbnr_workspace_bytes(self.grid, self.vset, o)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        o.dev_buffer = ctypes.c_void_p(self.workspace.data_ptr())
        o.dev_bytes = nbytes
        self.opts = o
        self.tau, self.dx = float(tau), float(dx)
        self.dt = float(dx if dt is None else dt)
        self.ctx = lbnr_create(self.grid, self.vset, self.tau, self.dx, self.dt, o)
        self.streaming = library().lbnr_streaming(self.ctx)
        self.variant = 0

    def init(self, fields):
        a = fields if not isinstance(fields, np.ndarray) else np.ascontiguousarray(
            fields, dtype=np.float64).reshape(16, self.cells)
        lbnr_init(self.ctx, a)

    def step(self, n=1):
        lbnr_step(self.ctx, n)

    @property
    def variants(self):
        return [lbnr_variant_name(self.ctx, v) for v in range(lbnr_num_variants(self.ctx))]

    def set_variant(self, v):
        lbnr_set_variant(self.ctx, v)
        self.variant = v

    def set_fluid(self, rho0, w, t0=1.0):
        """Perfect fluid at rest: density rho0 (t0/t)^2, pressure w rho, the
        state after n steps at t = t0 + n dt (call before init)."""
        lbnr_set_fluid(self.ctx, rho0, w, t0)

    def set_shift(self, beta):
        """Constant shift beta^i = (bx, by, bz) (call before init)."""
        bx, by, bz = (float(v) for v in beta)
        lbnr_set_shift(self.ctx, bx, by, bz)

    def set_shift_field(self, field):
        """Static shift field beta^i(x), [3][nz][ny][nx] or [3][cells], or
        None to remove it (call before init)."""
        if field is None:
            lbnr_set_shift_field(self.ctx, None)
            return
        f = np.ascontiguousarray(np.asarray(field, dtype=np.float64).reshape(3, self.cells))
        lbnr_set_shift_field(self.ctx, f)

    def step_timed(self, n=1):
        return lbnr_step_timed(self.ctx, n)

    def moments(self, out=None):
        out = np.empty((16, self.cells)) if out is None else out
        lbnr_moments(self.ctx, out)
        return out

    def constraints(self):
        out = np.empty(22)
        lbnr_constraints(self.ctx, out)
        return out

    def distributions(self):
        out = np.empty((16, self.Q, self.cells))
        lbnr_get_distributions(self.ctx, out)
        return out

    def cells_distributions(self, cells):
        out = np.empty((len(cells), 16, self.Q))
        lbnr_get_cells(self.ctx, cells, out)
        return out

    def set_distributions(self, f):
        lbnr_set_distributions(self.ctx, np.ascontiguousarray(f, dtype=np.float64))

    def status(self):
        lbnr_status(self.ctx)

    def lagged(self):
        """LAG: the lagged fields [7][cells] (alpha, gamma_ij) the next step
        differentiates."""
        out = np.empty((7, self.cells))
        lbnr_get_lagged(self.ctx, out)
        return out

    def set_lagged(self, prev):
        lbnr_set_lagged(self.ctx, np.ascontiguousarray(np.asarray(prev, dtype=np.float64)
                                                       .reshape(7, self.cells)))

    @property
    def deriv_mode(self):
        return library().lbnr_deriv_mode(self.ctx)

    @property
    def steps_done(self):
        return lbnr_steps_done(self.ctx)

    def close(self):
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            lbnr_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many independent 1D/2D lattices advanced by one persistent launch.

    runs: sequence of dicts with keys vset (1 or 2), shape (nx, ny), tau, dx,
    steps (per run() call) and optionally slicing. storage as for Lattice.
    """

    def __init__(self, runs, storage="dev_f32", block=256, ctas_per_sm=0, sources_on=True,
                 wait_limit_ns=2_000_000_000, drop_arrival_run=-1, replan=False, stream=None,
                 device=None, deriv_mode=LBNR_DERIV_SYNC):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("lbnr needs a CUDA device; there is no CPU path")
        self.device = torch.device(device or "cuda")
        library()
        self.stream = stream or torch.cuda.current_stream(self.device)
        if self.stream.cuda_stream == 0:
            self.stream = torch.cuda.Stream(self.device)
        descs = []
        self.runs = []
        for r in runs:
            nx, ny = (tuple(r["shape"]) + (1,))[:2]
            d = RunDesc(int(r["vset"]), int(r.get("slicing", LBNR_HARMONIC)),
                        Grid(int(nx), int(ny), 1), float(r["tau"]), float(r["dx"]),
                        int(r["steps"]))
            descs.append(d)
            self.runs.append(dict(r, cells=int(nx) * int(ny), Q=Q_OF[int(r["vset"])]))
        o = lbnr_default_batch_opts()
        o.storage = int(STORAGE_NAMES.get(storage, storage))
        o.block = int(block)
        o.ctas_per_sm = int(ctas_per_sm)
        o.sources_on = int(bool(sources_on))
        o.cuda_stream = ctypes.c_void_p(self.stream.cuda_stream)
        o.wait_limit_ns = int(wait_limit_ns)
        o.test_drop_arrival_run = int(drop_arrival_run)
        o.replan = int(bool(replan))
        o.deriv_mode = {"sync": LBNR_DERIV_SYNC, "lag": LBNR_DERIV_LAG}.get(deriv_mode, deriv_mode)
        self.storage = o.storage
        self.b = lbnr_batch_create(descs, o)

    def __len__(self):
        return len(self.runs)

    def init(self, run, fields):
        a = np.ascontiguousarray(fields, dtype=np.float64).reshape(16, self.runs[run]["cells"])
        lbnr_batch_init(self.b, run, a)

    def configure(self, block, ctas_per_sm=0):
        lbnr_batch_configure(self.b, block, ctas_per_sm)

    def run(self, max_steps=-1):
        lbnr_batch_run(self.b, max_steps)

    def replan(self):
        lbnr_batch_replan(self.b)

    def status(self):
        return lbnr_batch_status(self.b, len(self.runs))

    def check(self):
        rc, per = self.status()
        _check(rc, batch=self.b)
        return per

    def distributions(self, run):
        r = self.runs[run]
        out = np.empty((16, r["Q"], r["cells"]))
        lbnr_batch_get_distributions(self.b, run, out)
        return out

    def plan(self):
        return lbnr_batch_plan(self.b, len(self.runs))

    def steps_done(self, run):
        return lbnr_batch_steps_done(self.b, run)

    def close(self):
        if getattr(self, "b", None) is not None and self.b.value:
            lbnr_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ADLattice:
    """The 37-field scheme with independently evolved A_k and D_kij (the
    original Bona-Masso formulation; lbnr_ad_* in include/lbnr.h): the 16
    fields, then A_x A_y A_z, then D_kij at 19 + 6 k + pair. Ping-pong,
    storage "f64" or "f32"."""

    NF = 37

    def __init__(self, vset, shape, tau, dx, slicing=LBNR_HARMONIC, storage="f64", stream=None):
        lib = library()
        self.vset, self.shape = int(vset), tuple(int(v) for v in shape)
        self.cells = self.shape[0] * self.shape[1] * self.shape[2]
        self.Q = {1: 3, 2: 9, 3: 19}[self.vset]
        st = {"f64": LBNR_F64, "f32": LBNR_F32}[storage]
        self.ctx = ctypes.c_void_p()
        g = Grid(*self.shape)
        sp = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
        _check(lib.lbnr_ad_create(ctypes.byref(g), self.vset, float(tau), float(dx), float(dx),
                                  int(slicing), st, sp, ctypes.byref(self.ctx)), ad=None)
        self.form = 0 if storage == "f64" else 5

    @property
    def forms(self):
        """Launch forms: thread blocks per SM the registers are sized for."""
        lib = library()
        names = {0: "smem-staged, 1 lane/cell", -1: "smem-staged, 2 lanes/cell"}
        return [names.get(b, f"{b} blocks/SM") for b in
                (lib.lbnr_ad_form_blocks(i) for i in range(lib.lbnr_ad_num_forms()))]

    def set_form(self, form):
        _check(library().lbnr_ad_set_form(self.ctx, int(form)), ad=self.ctx)
        self.form = int(form)

    def init(self, fields):
        f = np.ascontiguousarray(np.asarray(fields, dtype=np.float64)).reshape(-1, self.cells)
        _check(library().lbnr_ad_init(self.ctx, _dptr(f), f.shape[0]), ad=self.ctx)

    def step(self, n=1):
        _check(library().lbnr_ad_step(self.ctx, int(n)), ad=self.ctx)

    def step_timed(self, n=1):
        ms = ctypes.c_double()
        _check(library().lbnr_ad_step_timed(self.ctx, int(n), ctypes.byref(ms)), ad=self.ctx)
        return ms.value

    def moments(self):
        out = np.empty((self.NF, self.cells))
        _check(library().lbnr_ad_moments(self.ctx, _dptr(out)), ad=self.ctx)
        return out

    def status(self):
        _check(library().lbnr_ad_status(self.ctx), ad=self.ctx)

    def distributions(self):
        out = np.empty((self.NF, self.Q, self.cells))
        _check(library().lbnr_ad_get_distributions(self.ctx, _dptr(out)), ad=self.ctx)
        return out

    def set_distributions(self, f):
        f = np.ascontiguousarray(np.asarray(f, dtype=np.float64))
        _check(library().lbnr_ad_set_distributions(self.ctx, _dptr(f)), ad=self.ctx)

    def close(self):
        if self.ctx:
            library().lbnr_ad_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
