"""Python binding of the C ABI in ``include/swe.h`` (argument marshalling only).

Every step of the CSPH-TVD + Exner method runs in the CUDA kernels of the
in-tree library ``_lib/libswe.so``; this module converts numpy arrays or
torch CUDA tensors to pointers and status codes to exceptions.  There is no
CPU fallback: if the library cannot be built or loaded, ``load_library``
raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from . import build as _build

SWE_OK, SWE_EINVAL, SWE_ENOMEM, SWE_ECUDA, SWE_ENUMERIC, SWE_ETIMEOUT, SWE_ESTATE = range(7)
SWE_FP64, SWE_FP32 = 0, 1
SWE_HOST, SWE_DEVICE = 0, 1
STATUS_NAMES = {0: "SWE_OK", 1: "SWE_EINVAL", 2: "SWE_ENOMEM", 3: "SWE_ECUDA", 4: "SWE_ENUMERIC",
                5: "SWE_ETIMEOUT", 6: "SWE_ESTATE"}
HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "swe.h")


class SweError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("dx", ctypes.c_double), ("g", ctypes.c_double),
        ("cfl_K", ctypes.c_double), ("eps_wet", ctypes.c_double), ("dt_max", ctypes.c_double),
        ("psi", ctypes.c_double), ("sediment_on", ctypes.c_int), ("aj_mode", ctypes.c_int),
        ("A_J", ctypes.c_double), ("m_exp", ctypes.c_double), ("C_J", ctypes.c_double),
        ("d50", ctypes.c_double), ("s_rel", ctypes.c_double), ("C_Sh", ctypes.c_double),
        ("dt_literal_D", ctypes.c_int), ("precision", ctypes.c_int), ("hgs_skip", ctypes.c_int),
        ("tile_rows", ctypes.c_int), ("block_cols", ctypes.c_int), ("neg_tol", ctypes.c_double),
        ("bc", ctypes.c_int * 4),
    ]


_BC_SIDES = {"bc_w": 0, "bc_e": 1, "bc_s": 2, "bc_n": 3}
SWE_BC_WALL, SWE_BC_OPEN = 0, 1


def _set_param(p, key, value):
    """A swe_params field, or one side's boundary kind (bc_w, bc_e, bc_s, bc_n)."""
    if key in _BC_SIDES:
        p.bc[_BC_SIDES[key]] = int(value)
    elif hasattr(p, key):
        setattr(p, key, value)
    else:
        raise TypeError(f"unknown parameter {key}")


class Diag(ctypes.Structure):
    _fields_ = [
        ("t", ctypes.c_double), ("dt_last", ctypes.c_double), ("dt_next", ctypes.c_double),
        ("binding", ctypes.c_int), ("water_volume", ctypes.c_double),
        ("sediment_volume", ctypes.c_double), ("inflow_volume", ctypes.c_double),
        ("steps", ctypes.c_int64), ("wet_cells", ctypes.c_int64), ("active_tiles", ctypes.c_int32),
        ("total_tiles", ctypes.c_int32), ("tile_x", ctypes.c_int32), ("tile_y", ctypes.c_int32),
        ("status", ctypes.c_uint32), ("cells_computed", ctypes.c_uint64),
        ("cells_copied", ctypes.c_uint64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SurrogateStats(ctypes.Structure):
    _fields_ = [
        ("windows", ctypes.c_int64), ("surrogate_windows", ctypes.c_int64), ("plain_windows", ctypes.c_int64),
        ("judged", ctypes.c_int64), ("takeover_window", ctypes.c_int64),
        ("bed_time", ctypes.c_double), ("water_time", ctypes.c_double),
        ("err_last", ctypes.c_double), ("err_max", ctypes.c_double), ("err_mean", ctypes.c_double),
        ("err_zero_mean", ctypes.c_double), ("err_persist_mean", ctypes.c_double),
        ("err_linear_mean", ctypes.c_double), ("elev_err_max", ctypes.c_double), ("mode", ctypes.c_int),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_libs = {False: None, True: None}


def header_functions():
    """Names of the functions the public header declares."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:swe_status|const char \*)\s*(swe_\w+)\s*\(", txt, re.M)))


def load_library(build_if_missing: bool = True, checked: bool = False):
    """Loads (building it first if needed) the in-tree CUDA library; checked:
    its variant that tests every global index of the step kernel against its
    buffer (device status bit 8 on a skipped access)."""
    if _libs[checked] is not None:
        return _libs[checked]
    path = _build.LIB_CHECKED if checked else _build.LIB
    if build_if_missing and not _build.up_to_date(checked):
        path = _build.build(checked=checked)
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing; run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    vp, dp, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)
    H = ctypes.c_void_p
    sig = {
        "swe_params_default": [ctypes.POINTER(Params), ctypes.c_int, ctypes.c_int, ctypes.c_double],
        "swe_create": [ctypes.POINTER(Params), vp, ctypes.POINTER(H)],
        "swe_destroy": [H],
        "swe_set_manning": [H, dp, ctypes.c_int],
        "swe_set_sources": [H, ctypes.POINTER(ctypes.c_uint8), dp, dp, ctypes.c_int],
        "swe_set_bed_source": [H, dp],
        "swe_set_rain": [H, dp],
        "swe_set_infiltration": [H, dp],
        "swe_set_state": [H, dp, dp, dp, dp],
        "swe_set_state_ex": [H, vp, vp, vp, vp, ctypes.c_int, ctypes.c_int],
        "swe_get_state": [H, dp, dp, dp, dp],
        "swe_get_state_ex": [H, vp, vp, vp, vp, ctypes.c_int, ctypes.c_int],
        "swe_step": [H, dp],
        "swe_advance": [H, ctypes.c_double, i64p],
        "swe_run_steps": [H, ctypes.c_int64],
        "swe_sync": [H],
        "swe_get_time": [H, dp],
        "swe_set_time": [H, ctypes.c_double],
        "swe_get_diag": [H, ctypes.POINTER(Diag)],
        "swe_get_census": [H, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int),
                           ctypes.POINTER(ctypes.c_int)],
        "swe_step_noalloc": [ctypes.POINTER(Params), ctypes.c_double, vp, vp, vp, dp],
    }
    sig.update({
        "swe_ensemble_create": [ctypes.c_int, ctypes.POINTER(Params), vp, ctypes.POINTER(vp)],
        "swe_ensemble_destroy": [vp],
        "swe_ensemble_member": [vp, ctypes.c_int, ctypes.POINTER(H)],
        "swe_ensemble_run": [vp, ctypes.c_int64],
        "swe_ensemble_autotune": [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
        "swe_autotune": [H, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
        "swe_ensemble_set_timeout": [vp, ctypes.c_double, ctypes.c_int],
    })
    sig.update({
        "swe_set_sediment": [H, ctypes.c_int],
        "swe_surrogate_create": [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, vp, ctypes.POINTER(vp)],
        "swe_surrogate_destroy": [vp],
        "swe_surrogate_set_norm": [vp, ctypes.POINTER(ctypes.c_float)],
        "swe_surrogate_set_loss": [vp, ctypes.c_int],
        "swe_surrogate_forward": [vp, vp, vp, ctypes.c_int],
        "swe_surrogate_train_step": [vp, vp, vp, ctypes.c_int, ctypes.c_float, ctypes.POINTER(ctypes.c_float)],
        "swe_surrogate_params": [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_float), ctypes.c_int],
        "swe_surrogate_grads": [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_float)],
        "swe_surrogate_buffer": [vp, ctypes.c_int, ctypes.POINTER(vp)],
        "swe_surrogate_pack_state": [vp, H, vp, ctypes.POINTER(ctypes.c_int)],
        "swe_surrogate_save_bed": [vp, H],
        "swe_surrogate_save_mid": [vp, H],
        "swe_surrogate_pack_target": [vp, H, vp],
        "swe_surrogate_apply": [vp, H],
        "swe_surrogate_run": [vp, H, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                              ctypes.POINTER(SurrogateStats)],
        "swe_nn_tc_selftest": [ctypes.c_int, ctypes.c_int, vp, vp, vp],
    })
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.swe_last_error.argtypes = [H]
    L.swe_last_error.restype = ctypes.c_char_p
    L.swe_signatures = dict(sig, swe_last_error=[H])
    _libs[checked] = L
    return L


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _is_torch(x):
    return type(x).__module__.startswith("torch")


class Solver:
    """One CSPH-TVD + Exner grid on the current CUDA device.

    precision: 'fp32' (FP32 state, FP64 dt/accumulators) or 'fp64'.
    checked: run on the library's checked variant (every global index of
    the step kernel tested against its buffer; for tests).
    Other keyword arguments override fields of ``swe_params``."""

    @classmethod
    def _view(cls, handle, params, precision="fp32", lib=None):
        """A non-owning view of a handle owned elsewhere (an ensemble member)."""
        self = cls.__new__(cls)
        self._L = lib if lib is not None else load_library()
        self.params = params
        self.nx, self.ny, self.dx = params.nx, params.ny, params.dx
        self.precision = precision
        self._h = handle
        self._owned = False
        return self

    def __init__(self, nx, ny, dx, precision="fp32", stream=None, checked=False, **kw):
        L = load_library(checked=checked)
        self._L = L
        self._owned = True
        p = Params()
        self._check(L.swe_params_default(ctypes.byref(p), nx, ny, dx), None)
        p.precision = SWE_FP32 if precision == "fp32" else SWE_FP64
        for k, v in kw.items():
            _set_param(p, k, v)
        self.params = p
        self.nx, self.ny, self.dx = nx, ny, dx
        self.precision = precision
        h = ctypes.c_void_p()
        st = L.swe_create(ctypes.byref(p), ctypes.c_void_p(stream) if stream else None, ctypes.byref(h))
        if st != SWE_OK:
            raise SweError(st, "swe_create failed")
        self._h = h

    def _check(self, st, h="self"):
        if st != SWE_OK:
            msg = self._L.swe_last_error(self._h).decode() if h == "self" else ""
            raise SweError(st, msg)

    def close(self):
        if getattr(self, "_h", None):
            if getattr(self, "_owned", True):
                self._L.swe_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ inputs
    def set_manning(self, n, block=0):
        n = np.ascontiguousarray(n, dtype=np.float64)
        self._check(self._L.swe_set_manning(self._h, _ptr(n), int(block)))

    def set_sources(self, mask, t=None, Q=None):
        if mask is None:
            self._check(self._L.swe_set_sources(self._h, None, None, None, 0))
            return
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        assert m.shape == (self.ny, self.nx)
        t = np.ascontiguousarray(t, dtype=np.float64)
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        self._check(self._L.swe_set_sources(self._h, m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                            _ptr(t), _ptr(Q), len(t)))

    def set_rain(self, sigma):
        """Per-cell water source in m/s ([ny, nx] or scalar), None to remove."""
        if sigma is None:
            self._check(self._L.swe_set_rain(self._h, None))
        else:
            s = np.ascontiguousarray(np.broadcast_to(sigma, (self.ny, self.nx)), dtype=np.float64)
            self._check(self._L.swe_set_rain(self._h, _ptr(s)))

    def set_infiltration(self, beta):
        """Per-cell infiltration rate in m/s ([ny, nx] or scalar), None to remove."""
        if beta is None:
            self._check(self._L.swe_set_infiltration(self._h, None))
        else:
            s = np.ascontiguousarray(np.broadcast_to(beta, (self.ny, self.nx)), dtype=np.float64)
            self._check(self._L.swe_set_infiltration(self._h, _ptr(s)))

    def set_bed_source(self, q):
        if q is None:
            self._check(self._L.swe_set_bed_source(self._h, None))
        else:
            q = np.ascontiguousarray(q, dtype=np.float64)
            self._check(self._L.swe_set_bed_source(self._h, _ptr(q)))

    def set_state(self, H, Hu, Hv, b):
        """Host numpy arrays (float64 or float32) or torch CUDA tensors."""
        arrs = [H, Hu, Hv, b]
        if _is_torch(H):
            import torch
            ts = [a.contiguous() for a in arrs]
            dt = SWE_FP64 if ts[0].dtype == torch.float64 else SWE_FP32
            ts = [a.to(ts[0].dtype) for a in ts]
            torch.cuda.current_stream().synchronize()
            self._check(self._L.swe_set_state_ex(self._h, *[ctypes.c_void_p(a.data_ptr()) for a in ts],
                                                 dt, SWE_DEVICE))
            return
        dtype = np.float32 if np.asarray(H).dtype == np.float32 else np.float64
        arrs = [np.ascontiguousarray(a, dtype=dtype) for a in arrs]
        for a in arrs:
            assert a.shape == (self.ny, self.nx), a.shape
        self._check(self._L.swe_set_state_ex(self._h, *[ctypes.c_void_p(a.ctypes.data) for a in arrs],
                                             SWE_FP64 if dtype == np.float64 else SWE_FP32, SWE_HOST))

    def get_state(self, dtype=np.float64, out=None):
        """Host copy of (H, Hu, Hv, b); `out` may supply four C-contiguous arrays."""
        if out is None:
            out = [np.empty((self.ny, self.nx), dtype=dtype) for _ in range(4)]
        dtype = out[0].dtype
        self._check(self._L.swe_get_state_ex(self._h, *[ctypes.c_void_p(a.ctypes.data) for a in out],
                                             SWE_FP64 if dtype == np.float64 else SWE_FP32, SWE_HOST))
        return out

    def get_state_device(self, tensors):
        import torch
        dt = SWE_FP64 if tensors[0].dtype == torch.float64 else SWE_FP32
        self._check(self._L.swe_get_state_ex(self._h, *[ctypes.c_void_p(a.data_ptr()) for a in tensors],
                                             dt, SWE_DEVICE))

    # ------------------------------------------------------------ stepping
    def step(self):
        dt = ctypes.c_double(0.0)
        self._check(self._L.swe_step(self._h, ctypes.byref(dt)))
        return dt.value

    def advance(self, t_end):
        n = ctypes.c_int64(0)
        self._check(self._L.swe_advance(self._h, float(t_end), ctypes.byref(n)))
        return n.value

    def run_steps(self, n):
        self._check(self._L.swe_run_steps(self._h, int(n)))

    def sync(self):
        self._check(self._L.swe_sync(self._h))

    @property
    def t(self):
        v = ctypes.c_double(0.0)
        self._check(self._L.swe_get_time(self._h, ctypes.byref(v)))
        return v.value

    def set_sediment(self, on):
        self._check(self._L.swe_set_sediment(self._h, int(bool(on))))

    def set_time(self, t):
        self._check(self._L.swe_set_time(self._h, float(t)))

    def diag(self):
        d = Diag()
        self._check(self._L.swe_get_diag(self._h, ctypes.byref(d)))
        return d.as_dict()

    def census(self):
        tx, ty = ctypes.c_int(0), ctypes.c_int(0)
        self._check(self._L.swe_get_census(self._h, None, ctypes.byref(tx), ctypes.byref(ty)))
        out = np.zeros((ty.value, tx.value), dtype=np.int32)
        self._check(self._L.swe_get_census(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                           ctypes.byref(tx), ctypes.byref(ty)))
        return out

    @property
    def tile(self):
        d = self.diag()
        return d["tile_x"], d["tile_y"]

    def autotune(self, trial_steps=5):
        """Times the candidate block shapes on the current state, keeps the
        fastest and restores the state and time; returns (block_cols, tile_rows)."""
        bw, th = ctypes.c_int(0), ctypes.c_int(0)
        self._check(self._L.swe_autotune(self._h, int(trial_steps), ctypes.byref(bw), ctypes.byref(th)))
        return bw.value, th.value


class Ensemble:
    """Independent scenarios advanced together by one persistent launch per
    run call (swe_ensemble_* in include/swe.h).  specs: list of dicts with
    nx, ny, dx and optional swe_params fields.  checked: the library's
    checked variant (see Solver)."""

    def __init__(self, specs, stream=None, block_cols=0, tile_rows=0, checked=False):
        L = load_library(checked=checked)
        self._L = L
        n = len(specs)
        arr = (Params * n)()
        for k, sp in enumerate(specs):
            p = arr[k]
            st = L.swe_params_default(ctypes.byref(p), sp["nx"], sp["ny"], sp["dx"])
            if st != SWE_OK:
                raise SweError(st, "swe_params_default")
            p.precision = SWE_FP32
            p.block_cols = block_cols
            p.tile_rows = tile_rows
            for key, v in sp.items():
                if key in ("nx", "ny", "dx"):
                    continue
                _set_param(p, key, v)
        h = ctypes.c_void_p()
        st = L.swe_ensemble_create(n, arr, ctypes.c_void_p(stream) if stream else None, ctypes.byref(h))
        if st != SWE_OK:
            raise SweError(st, "swe_ensemble_create failed")
        self._h = h
        self._params = arr
        self.members = []
        for k in range(n):
            mh = ctypes.c_void_p()
            self._check(L.swe_ensemble_member(self._h, k, ctypes.byref(mh)))
            self.members.append(Solver._view(mh, arr[k], lib=L))

    def _check(self, st):
        if st != SWE_OK:
            raise SweError(st, "ensemble call failed")

    def run(self, nsteps):
        self._check(self._L.swe_ensemble_run(self._h, int(nsteps)))

    def autotune(self, trial_steps=5):
        bw, th = ctypes.c_int(0), ctypes.c_int(0)
        self._check(self._L.swe_ensemble_autotune(self._h, int(trial_steps), ctypes.byref(bw), ctypes.byref(th)))
        return bw.value, th.value

    def set_timeout(self, seconds, extra_arrivals=0):
        self._check(self._L.swe_ensemble_set_timeout(self._h, float(seconds), int(extra_arrivals)))

    def close(self):
        if getattr(self, "_h", None):
            for m in self.members:
                m._h = None
            self._L.swe_ensemble_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Surrogate:
    """The learned bed surrogate (swe_surrogate_* in include/swe.h).  Tensors
    passed in are torch CUDA tensors; nothing is computed in Python."""

    CIN = (8, 32, 32, 32, 32, 32)
    NOUT = (32, 32, 32, 32, 32, 1)

    def __init__(self, tile=1024, max_batch=4, seed=0, stream=None):
        L = load_library()
        self._L = L
        self.tile, self.max_batch = tile, max_batch
        h = ctypes.c_void_p()
        st = L.swe_surrogate_create(tile, max_batch, seed, ctypes.c_void_p(stream) if stream else None, ctypes.byref(h))
        if st != SWE_OK:
            raise SweError(st, "swe_surrogate_create failed")
        self._h = h

    def _check(self, st):
        if st != SWE_OK:
            raise SweError(st, "surrogate call failed")

    @staticmethod
    def _p(t):
        return ctypes.c_void_p(t.data_ptr())

    def set_norm(self, norm):
        """norm: H mean, H std, b mean, b std, velocity scale, transport
        scale, output unit (m of bed change), first-step scale (unit / K)."""
        assert len(norm) == 8
        a = (ctypes.c_float * 8)(*[float(x) for x in norm])
        self._check(self._L.swe_surrogate_set_norm(self._h, a))

    def set_loss(self, kind):
        """'mse' (default) or 'l1'."""
        self._check(self._L.swe_surrogate_set_loss(self._h, {"mse": 0, "l1": 1}[kind]))

    def forward(self, X, out, B):
        self._check(self._L.swe_surrogate_forward(self._h, self._p(X), self._p(out), int(B)))

    def train_step(self, X, target, B, lr):
        loss = ctypes.c_float(0.0)
        self._check(self._L.swe_surrogate_train_step(self._h, self._p(X), self._p(target), int(B), float(lr),
                                                     ctypes.byref(loss)))
        return loss.value

    def _size(self, layer):
        return self.NOUT[layer] * 9 * self.CIN[layer] + self.NOUT[layer]

    def params(self, layer):
        a = np.zeros(self._size(layer), dtype=np.float32)
        self._check(self._L.swe_surrogate_params(self._h, layer, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), 0))
        n = self.NOUT[layer]
        return a[:-n].reshape(n, -1).copy(), a[-n:].copy()

    def set_params(self, layer, Wm, b):
        a = np.concatenate([np.asarray(Wm, np.float32).ravel(), np.asarray(b, np.float32).ravel()])
        assert a.size == self._size(layer)
        self._check(self._L.swe_surrogate_params(self._h, layer, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), 1))

    def grads(self, layer):
        a = np.zeros(self._size(layer), dtype=np.float32)
        self._check(self._L.swe_surrogate_grads(self._h, layer, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        n = self.NOUT[layer]
        return a[:-n].reshape(n, -1).copy(), a[-n:].copy()

    def buffer_ptr(self, index):
        p = ctypes.c_void_p()
        self._check(self._L.swe_surrogate_buffer(self._h, index, ctypes.byref(p)))
        return p.value

    def pack_state(self, solver, X):
        b = ctypes.c_int(0)
        self._check(self._L.swe_surrogate_pack_state(self._h, solver._h, self._p(X), ctypes.byref(b)))
        return b.value

    def save_bed(self, solver):
        self._check(self._L.swe_surrogate_save_bed(self._h, solver._h))

    def save_mid(self, solver):
        """The bed after the window's first coupled step (channels 5 and 6)."""
        self._check(self._L.swe_surrogate_save_mid(self._h, solver._h))

    def pack_target(self, solver, target):
        self._check(self._L.swe_surrogate_pack_target(self._h, solver._h, self._p(target)))

    def apply(self, solver):
        self._check(self._L.swe_surrogate_apply(self._h, solver._h))

    def run(self, solver, nwindows, K=50, f=25, judge_every=20, bound=0.5, stats=None):
        st = stats if stats is not None else SurrogateStats()
        self._check(self._L.swe_surrogate_run(self._h, solver._h, int(nwindows), int(K), int(f), int(judge_every),
                                              float(bound), ctypes.byref(st)))
        return st

    def close(self):
        if getattr(self, "_h", None):
            self._L.swe_surrogate_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

