"""Python access to the FP64 CPU oracle (``lbnr_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this module; the product library does
not, and it shares no code with the CUDA path.

The oracle follows the lattice Boltzmann model of Ilseven & Mendoza
(arXiv:1505.02037): Eq. (numlb) with the equilibria and source distributions
of Eqs. (alfa)-(ekstsor), the moment rule rho = sum f + dt S / 2, the
Bona-Masso right-hand sides of Sec. "Bona-Masso evolution equations" and the
ADM constraints of Sec. "3+1 ADM formalism". The C file lists every reading
of a passage the paper leaves open.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbnr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblbnr_oracle.so")
_lock = threading.Lock()
_lib = None

NF = 16
NF_AD = 37  # with independently evolved A_k (3) and D_kij (18)
Q_OF = {1: 3, 2: 9, 3: 19}
VSET_NAMES = {"D1Q3": 1, "D2Q9": 2, "D3Q19": 3}


class Params(ctypes.Structure):
    _fields_ = [
        ("vset", ctypes.c_int32),
        ("slicing", ctypes.c_int32),
        ("sources_on", ctypes.c_int32),
        ("deriv_mode", ctypes.c_int32),
        ("nx", ctypes.c_int64),
        ("ny", ctypes.c_int64),
        ("nz", ctypes.c_int64),
        ("dx", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("tau", ctypes.c_double),
        ("t", ctypes.c_double),
        ("fluid_on", ctypes.c_int32),
        ("pad2", ctypes.c_int32),
        ("fluid_rho0", ctypes.c_double),
        ("fluid_w", ctypes.c_double),
        ("fluid_t0", ctypes.c_double),
        ("beta", ctypes.c_double * 3),
        ("beta_field", ctypes.POINTER(ctypes.c_double)),
    ]


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc (no FMA contraction, optional OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            pp = ctypes.POINTER(Params)
            L.orc_vset.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), dp]
            L.orc_vset.restype = ctypes.c_int
            L.orc_bm_point.argtypes = [ctypes.c_double, dp, dp, dp, dp, dp, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_double, dp, dp, dp, dp]
            L.orc_bm_point.restype = None
            for name in ("orc_init", "orc_step", "orc_moments"):
                getattr(L, name).argtypes = [pp, dp, dp]
                getattr(L, name).restype = ctypes.c_int
            L.orc_run.argtypes = [pp, dp, dp, ctypes.c_int64]
            for name in ("orc_ad_init", "orc_ad_init37", "orc_ad_step", "orc_ad_moments"):
                getattr(L, name).argtypes = [pp, dp, dp]
                getattr(L, name).restype = ctypes.c_int
            L.orc_ad_run.argtypes = [pp, dp, dp, ctypes.c_int64]
            L.orc_ad_run.restype = ctypes.c_int
            L.orc_run.restype = ctypes.c_int
            L.orc_step_cells.argtypes = [pp, dp, ctypes.c_int64,
                                         ctypes.POINTER(ctypes.c_int64), dp]
            L.orc_step_cells.restype = ctypes.c_int
            L.orc_constraint_fields.argtypes = [pp, dp, dp]
            L.orc_constraint_fields.restype = ctypes.c_int
            L.orc_constraints.argtypes = [pp, dp, dp]
            L.orc_constraints.restype = ctypes.c_int
            L.orc_step_lag.argtypes = [pp, dp, dp, dp, dp]
            L.orc_step_lag.restype = ctypes.c_int
            L.orc_moments_lag.argtypes = [pp, dp, dp, dp]
            L.orc_moments_lag.restype = ctypes.c_int
            L.orc_constraints_lag.argtypes = [pp, dp, dp, dp]
            L.orc_constraints_lag.restype = ctypes.c_int
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class OracleError(RuntimeError):
    pass


def _check(rc: int, what: str):
    if rc == -4:
        raise FloatingPointError(f"oracle {what}: non-finite value")
    if rc != 0:
        raise OracleError(f"oracle {what} failed with code {rc}")


def velocity_set(vset: int):
    """(c[Q,3] int, w[Q] float) as tabulated in the oracle."""
    c = (ctypes.c_int * 57)()
    w = np.zeros(19)
    Q = lib().orc_vset(vset, c, _dp(w))
    if Q < 0:
        raise OracleError("unknown velocity set")
    return np.array(c[: 3 * Q]).reshape(Q, 3), w[:Q].copy()


def bm_point(alpha, g6, K6, V3, A3, D18, slicing=1, rho=0.0, P=0.0):
    """Pointwise lambda^k_ij [3,6], S_ij [6], Omega_k [3], lapse source; rho
    and P are the density and pressure of a fluid at rest (0: vacuum)."""
    g6, K6, V3, A3, D18 = (np.ascontiguousarray(np.asarray(v, dtype=np.float64))
                           for v in (g6, K6, V3, A3, D18))
    lam = np.zeros(18)
    S = np.zeros(6)
    Om = np.zeros(3)
    Sa = ctypes.c_double(0)
    lib().orc_bm_point(float(alpha), _dp(g6), _dp(K6), _dp(V3), _dp(A3), _dp(D18.reshape(-1)),
                       int(slicing), float(rho), float(P), _dp(lam), _dp(S), _dp(Om),
                       ctypes.byref(Sa))
    return lam.reshape(3, 6), S, Om, Sa.value


class Oracle:
    """One lattice configuration: vset 1/2/3, grid (nx, ny, nz), tau (the
    dimensionless tau/dt), dx = dt, slicing 0/1/2, sources on/off.

    fluid = (rho0, w, t0): a perfect fluid at rest with density
    rho0 (t0/t)^2 and pressure w rho (Sec. "Expansion of flat universe"). The
    calls then take the time t of the state they read (default t0; run()
    advances it by dt per step).

    shift = (bx, by, bz): a constant, uniform shift beta^i (Sec. "Bona-Masso
    evolution equations" with B = 0); default zero. shift_field: a static
    shift field beta^i(x), [3][nz][ny][nx] (or [3][cells]), added to shift;
    its B_k^i = d_k beta^i / 2 come from central differences.

    deriv_mode: the time level of A_k and D_kij (the paper is silent): 0 SYNC,
    this step's rho~ (reading R5); 1 LAG, the previous step's corrected alpha
    and gamma (R17: the state is then (f, prev), prev [7][cells], see
    lag_init / step_lag); 2 FIXED, the moment rule solved as an equation by
    fixed-point iteration (R18)."""

    def __init__(self, vset, shape, tau, dx, dt=None, slicing=1, sources_on=True, fluid=None,
                 shift=None, shift_field=None, deriv_mode=0):
        nx, ny, nz = shape
        self.vset = int(vset)
        self.Q = Q_OF[self.vset]
        self.shape = (int(nx), int(ny), int(nz))
        self.cells = nx * ny * nz
        self.p = Params(self.vset, int(slicing), int(bool(sources_on)), int(deriv_mode), nx, ny,
                        nz, float(dx), float(dx if dt is None else dt), float(tau))
        self.t0 = 1.0
        if fluid is not None:
            rho0, w, t0 = fluid
            self.p.fluid_on, self.p.fluid_rho0, self.p.fluid_w = 1, float(rho0), float(w)
            self.p.fluid_t0 = self.t0 = float(t0)
        self.p.t = self.t0
        if shift is not None:
            for k in range(3):
                self.p.beta[k] = float(shift[k])
        self._beta_field = None
        if shift_field is not None:
            bf = np.ascontiguousarray(np.asarray(shift_field, dtype=np.float64).reshape(3, -1))
            if bf.shape[1] != self.cells:
                raise ValueError("shift_field must hold 3 x cells values")
            self._beta_field = bf  # kept alive: the C side holds a pointer
            self.p.beta_field = _dp(bf)

    def _at(self, t):
        self.p.t = self.t0 if t is None else float(t)

    def _f_shape(self):
        return (NF, self.Q, self.cells)

    def init(self, fields: np.ndarray, t=None) -> np.ndarray:
        self._at(t)
        fields = np.ascontiguousarray(fields, dtype=np.float64).reshape(NF, self.cells)
        f = np.zeros(self._f_shape())
        _check(lib().orc_init(ctypes.byref(self.p), _dp(fields), _dp(f)), "init")
        return f

    def step(self, f: np.ndarray, t=None) -> np.ndarray:
        self._at(t)
        f = np.ascontiguousarray(f, dtype=np.float64)
        out = np.zeros(self._f_shape())
        _check(lib().orc_step(ctypes.byref(self.p), _dp(f), _dp(out)), "step")
        return out

    def run(self, f: np.ndarray, n: int, t=None) -> np.ndarray:
        self._at(t)
        f = np.array(f, dtype=np.float64, order="C", copy=True)
        scratch = np.zeros_like(f)
        _check(lib().orc_run(ctypes.byref(self.p), _dp(f), _dp(scratch), int(n)), "run")
        return f

    def moments(self, f: np.ndarray, t=None) -> np.ndarray:
        self._at(t)
        f = np.ascontiguousarray(f, dtype=np.float64)
        out = np.zeros((NF, self.cells))
        _check(lib().orc_moments(ctypes.byref(self.p), _dp(f), _dp(out)), "moments")
        return out

    # --- lagged derivatives (deriv_mode 1, reading R17) ----------------------
    def lag_init(self, fields: np.ndarray, t=None):
        """(f, prev): the initial distributions (as init) and the lagged fields
        of the first step, the initial alpha and gamma [7][cells]."""
        fields = np.ascontiguousarray(fields, dtype=np.float64).reshape(NF, self.cells)
        return self.init(fields, t), np.ascontiguousarray(fields[:7].copy())

    def step_lag(self, f: np.ndarray, prev: np.ndarray, t=None):
        """One step from (f, prev); returns the next (f, prev)."""
        self._at(t)
        f = np.ascontiguousarray(f, dtype=np.float64)
        prev = np.ascontiguousarray(prev, dtype=np.float64).reshape(7, self.cells)
        out = np.zeros(self._f_shape())
        pout = np.zeros((7, self.cells))
        _check(lib().orc_step_lag(ctypes.byref(self.p), _dp(f), _dp(prev), _dp(out), _dp(pout)),
               "step_lag")
        return out, pout

    def run_lag(self, f: np.ndarray, prev: np.ndarray, n: int, t=None):
        """n steps from (f, prev); the state's time advances by dt per step."""
        t0 = self.t0 if t is None else float(t)
        for i in range(int(n)):
            f, prev = self.step_lag(f, prev, t0 + i * self.p.dt)
        return f, prev

    def moments_lag(self, f: np.ndarray, prev: np.ndarray, t=None) -> np.ndarray:
        self._at(t)
        f = np.ascontiguousarray(f, dtype=np.float64)
        prev = np.ascontiguousarray(prev, dtype=np.float64).reshape(7, self.cells)
        out = np.zeros((NF, self.cells))
        _check(lib().orc_moments_lag(ctypes.byref(self.p), _dp(f), _dp(prev), _dp(out)),
               "moments_lag")
        return out

    def constraints_lag(self, f: np.ndarray, prev: np.ndarray) -> np.ndarray:
        f = np.ascontiguousarray(f, dtype=np.float64)
        prev = np.ascontiguousarray(prev, dtype=np.float64).reshape(7, self.cells)
        out = np.zeros(22)
        _check(lib().orc_constraints_lag(ctypes.byref(self.p), _dp(f), _dp(prev), _dp(out)),
               "constraints_lag")
        return out

    def step_cells(self, f: np.ndarray, cells, t=None) -> np.ndarray:
        self._at(t)
        f = np.ascontiguousarray(f, dtype=np.float64)
        idx = np.ascontiguousarray(np.asarray(cells, dtype=np.int64))
        out = np.zeros((len(idx), NF, self.Q))
        _check(lib().orc_step_cells(ctypes.byref(self.p), _dp(f), len(idx),
                                    idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                    _dp(out)), "step_cells")
        return out

    def constraint_fields(self, rho: np.ndarray) -> np.ndarray:
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(NF, self.cells)
        out = np.zeros((self.cells, 7))
        _check(lib().orc_constraint_fields(ctypes.byref(self.p), _dp(rho), _dp(out)),
               "constraint_fields")
        return out

    def constraints(self, f: np.ndarray) -> np.ndarray:
        f = np.ascontiguousarray(f, dtype=np.float64)
        out = np.zeros(22)
        _check(lib().orc_constraints(ctypes.byref(self.p), _dp(f), _dp(out)), "constraints")
        return out

    # --- independently evolved A_k and D_kij (37 distribution sets) ---------
    def ad_init(self, fields: np.ndarray, t=None) -> np.ndarray:
        """fields: [16][cells] (A, D start as central differences) or
        [37][cells] (A, D given)."""
        self._at(t)
        fields = np.ascontiguousarray(fields, dtype=np.float64).reshape(-1, self.cells)
        f = np.zeros((NF_AD, self.Q, self.cells))
        fn = {NF: "orc_ad_init", NF_AD: "orc_ad_init37"}[fields.shape[0]]
        _check(getattr(lib(), fn)(ctypes.byref(self.p), _dp(fields), _dp(f)), "ad_init")
        return f

    def ad_step(self, f: np.ndarray, t=None) -> np.ndarray:
        self._at(t)
        f = np.ascontiguousarray(f, dtype=np.float64)
        out = np.zeros((NF_AD, self.Q, self.cells))
        _check(lib().orc_ad_step(ctypes.byref(self.p), _dp(f), _dp(out)), "ad_step")
        return out

    def ad_run(self, f: np.ndarray, n: int, t=None) -> np.ndarray:
        self._at(t)
        f = np.array(f, dtype=np.float64, order="C", copy=True)
        scratch = np.zeros_like(f)
        _check(lib().orc_ad_run(ctypes.byref(self.p), _dp(f), _dp(scratch), int(n)), "ad_run")
        return f

    def ad_moments(self, f: np.ndarray, t=None) -> np.ndarray:
        self._at(t)
        f = np.ascontiguousarray(f, dtype=np.float64)
        out = np.zeros((NF_AD, self.cells))
        _check(lib().orc_ad_moments(ctypes.byref(self.p), _dp(f), _dp(out)), "ad_moments")
        return out
