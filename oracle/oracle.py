"""ctypes wrapper around the FP64 C oracle (oracle/misr_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the CPU-baseline
leg of bench.py.  The CUDA library never imports or links this module.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

MAXK = 64
MAXPSF = 15
REG_BTV, REG_TIKHONOV = 0, 1
HV_EXACT, HV_FD = 0, 1
NORM_L2, NORM_L1 = 0, 1
DECIM_POINT, DECIM_BIN = 0, 1


class _Problem(C.Structure):
    _fields_ = [
        ("h", C.c_int), ("w", C.c_int), ("K", C.c_int), ("f", C.c_int),
        ("ty", C.c_int * MAXK), ("tx", C.c_int * MAXK),
        ("psf_size", C.c_int), ("psf", C.c_double * (MAXPSF * MAXPSF)),
        ("lambda_", C.c_double), ("btv_alpha", C.c_double), ("btv_w", C.c_int),
        ("eps", C.c_double), ("reg", C.c_int),
        ("data_norm", C.c_int), ("data_eps", C.c_double), ("decim", C.c_int),
        ("fy", C.c_double * MAXK), ("fx", C.c_double * MAXK),
        ("state_f32", C.c_int),
    ]


TRACE_FIELDS = ("E", "J_trial", "alpha", "delta", "mu", "lam", "Delta", "pn2", "rn2", "accept")


class _TraceRow(C.Structure):
    _fields_ = [(n, C.c_double) for n in TRACE_FIELDS]


_lib = None


def lib():
    global _lib
    if _lib is None:
        # MISR_ORACLE_LIB lets the mutation test load a deliberately broken copy
        path = os.environ.get("MISR_ORACLE_LIB") or _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        pp = C.POINTER(_Problem)
        L.orc_init.argtypes = [pp, C.c_int, C.c_int, C.c_int, C.c_int, dp, dp, C.c_int,
                               C.c_double, C.c_double, C.c_int, C.c_double, C.c_int]
        L.orc_init.restype = C.c_int
        L.orc_threads.restype = C.c_int
        L.orc_set_data_norm.argtypes = [pp, C.c_int, C.c_double]
        L.orc_set_data_norm.restype = C.c_int
        L.orc_set_decimation.argtypes = [pp, C.c_int]
        L.orc_set_decimation.restype = C.c_int
        L.orc_set_state_f32.argtypes = [pp, C.c_int]
        L.orc_set_state_f32.restype = C.c_int
        for name in ("orc_forward", "orc_adjoint"):
            getattr(L, name).argtypes = [pp, C.c_int, dp, dp]
        L.orc_reg_value.argtypes = [pp, dp]
        L.orc_reg_value.restype = C.c_double
        L.orc_reg_grad.argtypes = [pp, dp, dp]
        L.orc_reg_hessvec.argtypes = [pp, dp, dp, dp]
        L.orc_reg_curvature.argtypes = [pp, dp, dp]
        L.orc_reg_curvature.restype = C.c_double
        L.orc_objective.argtypes = [pp, dp, dp]
        L.orc_objective.restype = C.c_double
        L.orc_gradient.argtypes = [pp, dp, dp, dp]
        L.orc_gradient.restype = C.c_double
        L.orc_hessvec.argtypes = [pp, dp, dp, dp, dp]
        L.orc_curvature.argtypes = [pp, dp, dp, dp]
        L.orc_curvature.restype = C.c_double
        L.orc_shift_add.argtypes = [pp, dp, dp]
        L.orc_log_convert.argtypes = [C.POINTER(C.c_ushort), C.c_long, C.c_double, dp]
        L.orc_scg.argtypes = [pp, dp, dp, C.c_int, C.c_int, dp, C.POINTER(_TraceRow)]
        L.orc_scg.restype = C.c_int
        _lib = L
    return _lib


def _d(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def threads() -> int:
    return int(lib().orc_threads())


class Problem:
    """One MISR problem: K LR frames of h x w, magnification f, shifts (dx, dy) in LR px."""

    def __init__(self, h, w, f, shifts, psf, lam=0.01, btv_alpha=0.4, btv_w=3, eps=1e-3,
                 reg=REG_BTV, data_norm=NORM_L2, data_eps=0.0, decimation=DECIM_POINT, state_f32=False):
        self.h, self.w, self.f = int(h), int(w), int(f)
        self.K = len(shifts)
        self.H, self.W = self.f * self.h, self.f * self.w
        sh = _f64(np.asarray(shifts, dtype=np.float64).reshape(-1))
        psf = _f64(psf)
        self._p = _Problem()
        rc = lib().orc_init(C.byref(self._p), self.h, self.w, self.K, self.f, _d(sh), _d(psf),
                            int(psf.shape[0]), float(lam), float(btv_alpha), int(btv_w),
                            float(eps), int(reg))
        if rc != 0:
            raise ValueError(f"orc_init failed ({rc})")
        if lib().orc_set_data_norm(C.byref(self._p), int(data_norm), float(data_eps)) != 0:
            raise ValueError("data norm: L2, or L1 with data_eps > 0")
        if lib().orc_set_decimation(C.byref(self._p), int(decimation)) != 0:
            raise ValueError("decimation: DECIM_POINT or DECIM_BIN")
        # FP32 storage of the SCG state (a sensitivity model; FP64 by default)
        if lib().orc_set_state_f32(C.byref(self._p), int(bool(state_f32))) != 0:
            raise ValueError("state_f32: a bool")
        self.data_norm = int(data_norm)

    @property
    def shifts_hr(self):
        return [(self._p.ty[k], self._p.tx[k]) for k in range(self.K)]

    @property
    def psf(self):
        s = self._p.psf_size
        return np.array(self._p.psf[: s * s]).reshape(s, s)

    def _x(self, x):
        x = _f64(x)
        assert x.shape == (self.H, self.W), x.shape
        return x

    def _y(self, y):
        y = _f64(y)
        assert y.shape == (self.K, self.h, self.w), y.shape
        return y

    def forward(self, k, x):
        x = self._x(x)
        out = np.empty((self.h, self.w))
        lib().orc_forward(C.byref(self._p), int(k), _d(x), _d(out))
        return out

    def forward_all(self, x):
        return np.stack([self.forward(k, x) for k in range(self.K)])

    def adjoint(self, k, e):
        e = _f64(e)
        assert e.shape == (self.h, self.w)
        out = np.empty((self.H, self.W))
        lib().orc_adjoint(C.byref(self._p), int(k), _d(e), _d(out))
        return out

    def reg_value(self, x):
        return float(lib().orc_reg_value(C.byref(self._p), _d(self._x(x))))

    def reg_grad(self, x):
        g = np.empty((self.H, self.W))
        lib().orc_reg_grad(C.byref(self._p), _d(self._x(x)), _d(g))
        return g

    def reg_hessvec(self, x, p):
        out = np.empty((self.H, self.W))
        lib().orc_reg_hessvec(C.byref(self._p), _d(self._x(x)), _d(self._x(p)), _d(out))
        return out

    def reg_curvature(self, x, p):
        return float(lib().orc_reg_curvature(C.byref(self._p), _d(self._x(x)), _d(self._x(p))))

    def objective(self, x, y):
        return float(lib().orc_objective(C.byref(self._p), _d(self._x(x)), _d(self._y(y))))

    def gradient(self, x, y):
        g = np.empty((self.H, self.W))
        J = lib().orc_gradient(C.byref(self._p), _d(self._x(x)), _d(self._y(y)), _d(g))
        return float(J), g

    def _y_or_null(self, y):
        # the frames enter the Hessian only through the L1 data term's weights
        if y is None:
            assert self.data_norm == NORM_L2, "the L1 data term's Hessian needs the frames"
            return None, None
        y = self._y(y)
        return y, _d(y)

    def hessvec(self, x, p, y=None):
        out = np.empty((self.H, self.W))
        keep, yp = self._y_or_null(y)
        lib().orc_hessvec(C.byref(self._p), _d(self._x(x)), yp, _d(self._x(p)), _d(out))
        return out

    def curvature(self, x, p, y=None):
        keep, yp = self._y_or_null(y)
        return float(lib().orc_curvature(C.byref(self._p), _d(self._x(x)), yp, _d(self._x(p))))

    def shift_add(self, y):
        out = np.empty((self.H, self.W))
        lib().orc_shift_add(C.byref(self._p), _d(self._y(y)), _d(out))
        return out

    def scg(self, y, x0, iters, hv_mode=HV_EXACT):
        x0 = self._x(x0)
        y = self._y(y)
        out = np.empty((self.H, self.W))
        tr = (_TraceRow * max(1, int(iters)))()
        n = lib().orc_scg(C.byref(self._p), _d(y), _d(x0), int(iters), int(hv_mode), _d(out), tr)
        trace = {k: np.array([getattr(tr[i], k) for i in range(n)]) for k in TRACE_FIELDS}
        return out, trace


def log_convert(counts, flat_field):
    c = np.ascontiguousarray(counts, dtype=np.uint16)
    out = np.empty(c.shape, dtype=np.float64)
    lib().orc_log_convert(c.ctypes.data_as(C.POINTER(C.c_ushort)), c.size, float(flat_field), _d(out))
    return out
