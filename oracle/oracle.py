"""Python handle on the FP64 CPU oracle (``swe_oracle.c``).

TEST INFRASTRUCTURE ONLY: the oracle is the slow reference definition of one
CSPH-TVD + Exner step (paper Sec. 2-3, Eq. 1-7, kernels K1-K8).  Only the test
suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this module.  It shares no code with the CUDA library.

``build()`` compiles the C source with gcc (``-ffp-contract=off`` so every
operation rounds exactly as written, ``-fopenmp`` for the tile loop).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field, asdict

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "swe_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liborc.so")


def build(force: bool = False) -> str:
    """Compile the oracle shared library in-tree; returns its path."""
    if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
        return _OUT
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    tmp = _OUT + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _OUT)
    return _OUT


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("dx", ctypes.c_double), ("g", ctypes.c_double), ("cfl_K", ctypes.c_double),
        ("eps_wet", ctypes.c_double), ("dt_max", ctypes.c_double), ("psi", ctypes.c_double),
        ("sediment_on", ctypes.c_int), ("aj_mode", ctypes.c_int),
        ("A_J", ctypes.c_double), ("m_exp", ctypes.c_double), ("C_J", ctypes.c_double),
        ("d50", ctypes.c_double), ("s_rel", ctypes.c_double), ("C_Sh", ctypes.c_double),
        ("dt_literal_D", ctypes.c_int), ("hgs_skip", ctypes.c_int),
        ("tile_x", ctypes.c_int), ("tile_y", ctypes.c_int),
        ("frozen_hydro", ctypes.c_int), ("neg_tol", ctypes.c_double),
        ("bc", ctypes.c_int * 4),
    ]


class _DtTerms(ctypes.Structure):
    _fields_ = [("vp", ctypes.c_double), ("vs", ctypes.c_double), ("J0max", ctypes.c_double)]


class _StepInfo(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("binding", ctypes.c_int),
                ("inflow_vol", ctypes.c_double), ("rain_vol", ctypes.c_double), ("outflow_vol", ctypes.c_double),
                ("infil_vol", ctypes.c_double),
                ("n_negative", ctypes.c_long), ("n_bad", ctypes.c_long), ("active_tiles", ctypes.c_long)]


@dataclass
class Params:
    """Model parameters; defaults are the readings for constants the paper leaves open."""
    nx: int
    ny: int
    dx: float = 1.0
    g: float = 9.81
    cfl_K: float = 0.4
    eps_wet: float = 1e-4
    dt_max: float = 1.0
    psi: float = 0.4
    sediment_on: int = 1
    aj_mode: int = 0
    A_J: float = 0.001
    m_exp: float = 2.0
    C_J: float = 2.0
    d50: float = 5e-4
    s_rel: float = 2.65
    C_Sh: float = 5.0
    dt_literal_D: int = 0
    hgs_skip: int = 1
    tile_x: int = 64
    tile_y: int = 64
    frozen_hydro: int = 0
    neg_tol: float = 1e-10
    bc_w: int = 0           # boundary kinds: 0 reflective wall, 1 open (zero-gradient)
    bc_e: int = 0
    bc_s: int = 0
    bc_n: int = 0

    def c(self) -> _Params:
        d = asdict(self)
        bc = [d.pop(k) for k in ("bc_w", "bc_e", "bc_s", "bc_n")]
        return _Params(**d, bc=(ctypes.c_int * 4)(*bc))


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        u8 = ctypes.POINTER(ctypes.c_uint8)
        L.orc_step.restype = ctypes.c_long
        L.orc_step.argtypes = [ctypes.POINTER(_Params), dp, dp, dp, dp, dp, u8, dp, dp, dp,
                               ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_double,
                               dp, dp, dp, dp, ctypes.POINTER(_StepInfo)]
        L.orc_step_rect.restype = ctypes.c_long
        L.orc_step_rect.argtypes = [ctypes.POINTER(_Params), dp, dp, dp, dp, dp, u8, dp, dp, dp,
                                    ctypes.c_double, ctypes.c_double,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    dp, dp, dp, dp, ctypes.POINTER(ctypes.c_long), dp, dp]
        L.orc_dt_terms.restype = ctypes.c_int
        L.orc_dt_terms.argtypes = [ctypes.POINTER(_Params), dp, dp, dp, dp, ctypes.POINTER(_DtTerms)]
        L.orc_dt.restype = ctypes.c_double
        L.orc_dt.argtypes = [ctypes.POINTER(_Params), ctypes.POINTER(_DtTerms), ctypes.POINTER(ctypes.c_int)]
        L.orc_census.restype = None
        L.orc_census.argtypes = [ctypes.POINTER(_Params), dp, u8, ctypes.POINTER(ctypes.c_int)]
        L.orc_hll.restype = ctypes.c_double
        L.orc_hll.argtypes = [ctypes.c_double] * 6
        L.orc_minmod.restype = ctypes.c_double
        L.orc_minmod.argtypes = [ctypes.c_double] * 2
        L.orc_hydro_integral.restype = ctypes.c_double
        L.orc_hydro_integral.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_double]
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_num_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, shape):
    a = np.ascontiguousarray(a, dtype=np.float64)
    assert a.shape == shape, (a.shape, shape)
    return a


def set_threads(n: int) -> int:
    """Sets the OpenMP thread count of the tile loop (n <= 0: leave); returns it."""
    return lib().orc_num_threads(int(n))


class Hydrograph:
    """Piecewise-linear inflow Q(t) [m^3/s] on the source-flagged cells."""

    def __init__(self, t, Q):
        self.t = np.ascontiguousarray(t, dtype=np.float64)
        self.Q = np.ascontiguousarray(Q, dtype=np.float64)

    def integral(self, ta, tb):
        return lib().orc_hydro_integral(len(self.t), _d(self.t), _d(self.Q), ta, tb)


@dataclass
class State:
    H: np.ndarray
    Hu: np.ndarray
    Hv: np.ndarray
    b: np.ndarray

    def copy(self):
        return State(self.H.copy(), self.Hu.copy(), self.Hv.copy(), self.b.copy())

    def arrays(self):
        return (self.H, self.Hu, self.Hv, self.b)


@dataclass
class StepInfo:
    dt: float
    binding: int
    inflow_vol: float
    n_negative: int
    n_bad: int
    active_tiles: int
    rain_vol: float = 0.0
    outflow_vol: float = 0.0
    infil_vol: float = 0.0


def _prep(p: Params, st: State, n, src, qb):
    shape = (p.ny, p.nx)
    H, Hu, Hv, b = (_f64(a, shape) for a in st.arrays())
    n = _f64(np.broadcast_to(n, shape), shape)
    srcp = None
    if src is not None:
        src = np.ascontiguousarray(src, dtype=np.uint8)
        assert src.shape == shape
        srcp = src.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    qbp = None
    if qb is not None:
        qb = _f64(qb, shape)
        qbp = _d(qb)
    return H, Hu, Hv, b, n, src, srcp, qb, qbp


def step(p: Params, st: State, n, src=None, qb=None, hydro: Hydrograph | None = None,
         t: float = 0.0, t_end: float = -1.0, rain=None, beta=None):
    """One full step (K1..K8).  rain: per-cell water source in m/s; beta:
    per-cell infiltration rate in m/s (each None or an array/scalar).
    Returns (new State, StepInfo)."""
    H, Hu, Hv, b, n, src, srcp, qb, qbp = _prep(p, st, n, src, qb)
    rainp = betap = None
    if rain is not None:
        rain = _f64(np.broadcast_to(rain, H.shape), H.shape)
        rainp = _d(rain)
    if beta is not None:
        beta = _f64(np.broadcast_to(beta, H.shape), H.shape)
        betap = _d(beta)
    out = [np.empty_like(H) for _ in range(4)]
    info = _StepInfo()
    pc = p.c()
    if hydro is not None:
        nk, tk, Qk = len(hydro.t), _d(hydro.t), _d(hydro.Q)
    else:
        nk, tk, Qk = 0, None, None
    lib().orc_step(ctypes.byref(pc), _d(H), _d(Hu), _d(Hv), _d(b), _d(n), srcp, qbp, rainp, betap,
                   nk, tk, Qk, t, t_end, *(_d(o) for o in out), ctypes.byref(info))
    return State(*out), StepInfo(info.dt, info.binding, info.inflow_vol, info.n_negative,
                                 info.n_bad, info.active_tiles, info.rain_vol, info.outflow_vol, info.infil_vol)


def step_rect(p: Params, st: State, n, dt: float, rect, src=None, qb=None, dHs: float = 0.0):
    """K2..K8 for the output rectangle (x0, y0, x1, y1) with a given dt.
    Returns the four output arrays of the rectangle and the bad-cell count."""
    x0, y0, x1, y1 = rect
    H, Hu, Hv, b, n, src, srcp, qb, qbp = _prep(p, st, n, src, qb)
    out = [np.zeros_like(H) for _ in range(4)]
    nneg = ctypes.c_long(0)
    pc = p.c()
    bad = lib().orc_step_rect(ctypes.byref(pc), _d(H), _d(Hu), _d(Hv), _d(b), _d(n), srcp, qbp, None, None,
                              dHs, dt, x0, y0, x1, y1, *(_d(o) for o in out), ctypes.byref(nneg), None, None)
    return [o[y0:y1, x0:x1].copy() for o in out], bad


def dt_terms(p: Params, st: State, n):
    H, Hu, Hv, b, n, *_ = _prep(p, st, n, None, None)
    t = _DtTerms()
    pc = p.c()
    lib().orc_dt_terms(ctypes.byref(pc), _d(H), _d(Hu), _d(Hv), _d(n), ctypes.byref(t))
    return t.vp, t.vs, t.J0max


def dt_from_terms(p: Params, vp: float, vs: float, J0max: float):
    t = _DtTerms(vp, vs, J0max)
    w = ctypes.c_int(0)
    pc = p.c()
    dt = lib().orc_dt(ctypes.byref(pc), ctypes.byref(t), ctypes.byref(w))
    return dt, w.value


def census(p: Params, H, src=None):
    shape = (p.ny, p.nx)
    H = _f64(H, shape)
    ntx = -(-p.nx // p.tile_x)
    nty = -(-p.ny // p.tile_y)
    out = np.zeros((nty, ntx), dtype=np.int32)
    srcp = None
    if src is not None:
        src = np.ascontiguousarray(src, dtype=np.uint8)
        srcp = src.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    pc = p.c()
    lib().orc_census(ctypes.byref(pc), _d(H), srcp, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return out


def hll(UL, UR, FL, FR, sL, sR):
    return lib().orc_hll(UL, UR, FL, FR, sL, sR)


def minmod(a, b):
    return lib().orc_minmod(a, b)


def run(p: Params, st: State, n, nsteps: int, src=None, qb=None, hydro=None, t: float = 0.0,
        t_end: float = -1.0, on_step=None, rain=None, beta=None):
    """Advances nsteps (or until t_end).  Returns (State, t, list of StepInfo)."""
    infos = []
    for _ in range(nsteps):
        if t_end > 0 and t >= t_end:
            break
        st, info = step(p, st, n, src=src, qb=qb, hydro=hydro, t=t, t_end=t_end, rain=rain, beta=beta)
        t = t_end if info.binding == 4 else t + info.dt   # a clipped step lands on t_end
        infos.append(info)
        if on_step is not None:
            on_step(st, t, info)
        if info.n_bad:
            raise FloatingPointError(f"oracle step produced {info.n_bad} bad cells")
    return st, t, infos
