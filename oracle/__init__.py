"""FP64 CPU oracle for the AC-OPF callbacks, polar and rectangular (ctypes wrapper of oracle.c).

TEST INFRASTRUCTURE ONLY. The oracle judges the CUDA library; only tests/,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it. It shares no code with ``paper_2510_12897_b300`` and is never on the
product path.

Parity status of each function (what pins it lives in tests/test_oracle_*.py):
  obj, grad      closed form of the quadratic cost; central differences
  cons           brute-force dense Y-bus on 3 buses; Newton power flow with zero
                 mismatch; textbook lossless-line and no-load flows
  jac            central differences (Richardson) of cons; sympy derivatives
                 of the pi-model at high precision
  hess           central differences of grad + J^T lambda; symmetry; sympy
  patterns       nnz closed forms; every structural nonzero found by
                 differences lies in the pattern
  bounds, cvio   closed forms on hand-built cases
  form="rect"    Newton power flow in rectangular voltages; equality with the
                 polar model at the same point; chain rule against the polar
                 Jacobian; trigonometric closed form of the angle rows; the
                 exact second-order expansion of the (quadratic) Lagrangian;
                 differences of cons and of grad + J^T lambda
  storage        state-of-charge rows zero along a recurrence-integrated
                 schedule; loss row zero at numpy's root of the loss balance
                 and its loss term r |I|^2 in complex arithmetic; balance rows
                 grow by ps, qs only; complementarity product; bounds; sizes;
                 differences of cons and of grad + J^T lambda
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liboracle.so")

_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (plain C99, no fast-math)."""
    src = os.path.join(_HERE, "oracle.c")
    hdr = os.path.join(_HERE, "oracle.h")
    if (not force and os.path.exists(LIB_PATH)
            and os.path.getmtime(LIB_PATH) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return LIB_PATH
    tmp = LIB_PATH + ".tmp"
    subprocess.check_call(["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-Wall", "-o", tmp,
                           src, "-lm"])
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class OraNet(ctypes.Structure):
    _fields_ = [
        ("nbus", ctypes.c_int32), ("nbranch", ctypes.c_int32), ("ngen", ctypes.c_int32),
        ("nload", ctypes.c_int32), ("nperiod", ctypes.c_int32), ("ref_bus", ctypes.c_int32),
        ("vmin", _f64p), ("vmax", _f64p), ("gs", _f64p), ("bs", _f64p),
        ("f", _i32p), ("t", _i32p),
        ("r", _f64p), ("x", _f64p), ("b", _f64p), ("tap", _f64p), ("shift", _f64p),
        ("rate_a", _f64p), ("angmin", _f64p), ("angmax", _f64p),
        ("gen_bus", _i32p),
        ("pmin", _f64p), ("pmax", _f64p), ("qmin", _f64p), ("qmax", _f64p),
        ("c2", _f64p), ("c1", _f64p), ("c0", _f64p),
        ("load_bus", _i32p), ("pd", _f64p), ("qd", _f64p),
        ("ramp_ratio", ctypes.c_double),
    ]


class OraStorage(ctypes.Structure):
    _fields_ = [
        ("nstor", ctypes.c_int32), ("bus", _i32p),
        ("energy_rating", _f64p), ("charge_rating", _f64p), ("discharge_rating", _f64p),
        ("thermal_rating", _f64p), ("eta_c", _f64p), ("eta_d", _f64p), ("r", _f64p),
        ("p_loss", _f64p), ("qmin", _f64p), ("qmax", _f64p), ("e_init", _f64p),
        ("dt", ctypes.c_double),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB_PATH)
        L.ora_create.restype = ctypes.c_void_p
        L.ora_create.argtypes = [ctypes.POINTER(OraNet), ctypes.c_int32, ctypes.c_double]
        L.ora_create2.restype = ctypes.c_void_p
        L.ora_create2.argtypes = [ctypes.POINTER(OraNet), ctypes.c_int32, ctypes.c_double, _f64p, ctypes.c_double]
        L.ora_create3.restype = ctypes.c_void_p
        L.ora_create3.argtypes = [ctypes.POINTER(OraNet), ctypes.c_int32, ctypes.c_double, _f64p, ctypes.c_double,
                                  ctypes.c_int32]
        L.ora_create4.restype = ctypes.c_void_p
        L.ora_create4.argtypes = [ctypes.POINTER(OraNet), ctypes.c_int32, ctypes.c_double, _f64p, ctypes.c_double,
                                  ctypes.c_int32, ctypes.POINTER(OraStorage), ctypes.c_int32]
        L.ora_destroy.argtypes = [ctypes.c_void_p]
        L.ora_error.restype = ctypes.c_char_p
        L.ora_dims.argtypes = [ctypes.c_void_p, _i64p, _i64p, _i64p, _i64p]
        L.ora_jac_pattern.argtypes = [ctypes.c_void_p, _i64p, _i64p]
        L.ora_hess_pattern.argtypes = [ctypes.c_void_p, _i64p, _i64p]
        L.ora_bounds.argtypes = [ctypes.c_void_p, _f64p, _f64p, _f64p, _f64p]
        L.ora_obj.restype = ctypes.c_double
        L.ora_obj.argtypes = [ctypes.c_void_p, _f64p]
        L.ora_obj_scale.restype = ctypes.c_double
        L.ora_obj_scale.argtypes = [ctypes.c_void_p, _f64p]
        L.ora_grad.argtypes = [ctypes.c_void_p, _f64p, _f64p]
        L.ora_cons.argtypes = [ctypes.c_void_p, _f64p, _f64p, _f64p]
        L.ora_jac.restype = ctypes.c_int
        L.ora_jac.argtypes = [ctypes.c_void_p, _f64p, _f64p, _f64p]
        L.ora_hess.restype = ctypes.c_int
        L.ora_hess.argtypes = [ctypes.c_void_p, _f64p, _f64p, ctypes.c_double, _f64p, _f64p]
        L.ora_cvio.argtypes = [ctypes.c_void_p, _f64p, _f64p, _f64p]
        _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a, typ):
    if a is None:
        return ctypes.cast(None, typ)
    return a.ctypes.data_as(typ)


class Oracle:
    """The oracle for one instance (a grid) or a batch (a list of grids).

    ``link_ratio > 0`` adds rows pg_s - pg_0 in [-ratio pmax, ratio pmax]
    tying every instance s >= 1 to instance 0 (``link_ratios``: one ratio
    per instance instead); ``reserve > 0`` adds per instance and period the
    row sum_g pg_g <= sum_g pmax_g - reserve * (total Pd). ``form``: "polar"
    (va, vm) or "rect" (vr, vi, with the angle and magnitude rows of the
    rectangular model). Grids carrying ``storage`` get the storage variables
    and rows; ``compl`` adds the complementarity rows sc sd <= 0.
    """

    def __init__(self, grids, link_ratio: float = 0.0, link_ratios=None, reserve: float = 0.0,
                 form: str = "polar", compl: bool = False):
        if form not in ("polar", "rect"):
            raise ValueError("form must be 'polar' or 'rect'")
        self.form = form
        if not isinstance(grids, (list, tuple)):
            grids = [grids]
        self.grids = list(grids)
        self._keep = []
        nets = (OraNet * len(grids))()
        for k, g in enumerate(grids):
            self._fill(nets[k], g)
        self._nets = nets
        lr = None
        if link_ratios is not None:
            lr = np.ascontiguousarray(link_ratios, dtype=np.float64)
            self._keep.append(lr)
        stor = None
        if any(getattr(g, "storage", None) is not None for g in grids):
            stor = (OraStorage * len(grids))()
            for k, g in enumerate(grids):
                self._fill_storage(stor[k], getattr(g, "storage", None))
        self._stor = stor
        self.ctx = lib().ora_create4(nets, len(grids), float(link_ratio),
                                     None if lr is None else lr.ctypes.data_as(_f64p), float(reserve),
                                     1 if form == "rect" else 0, stor, 1 if compl else 0)
        if not self.ctx:
            raise ValueError("oracle: " + lib().ora_error().decode())
        n, m, nj, nh = (ctypes.c_int64() for _ in range(4))
        lib().ora_dims(self.ctx, ctypes.byref(n), ctypes.byref(m), ctypes.byref(nj), ctypes.byref(nh))
        self.n, self.m, self.nnzj, self.nnzh = n.value, m.value, nj.value, nh.value

    def _fill(self, d, g):
        keep = self._keep

        def f(a):
            a = _f64(a)
            keep.append(a)
            return _p(a, _f64p)

        def i(a):
            a = _i32(a)
            keep.append(a)
            return _p(a, _i32p)

        d.nbus, d.nbranch, d.ngen = g.nbus, len(g.br_f), len(g.gen_bus)
        d.nload, d.nperiod, d.ref_bus = len(g.load_bus), g.load_pd.shape[0], g.ref_bus
        d.vmin, d.vmax, d.gs, d.bs = f(g.bus_vmin), f(g.bus_vmax), f(g.bus_gs), f(g.bus_bs)
        d.f, d.t = i(g.br_f), i(g.br_t)
        d.r, d.x, d.b = f(g.br_r), f(g.br_x), f(g.br_b)
        d.tap, d.shift = f(g.br_tap), f(g.br_shift)
        d.rate_a, d.angmin, d.angmax = f(g.br_rate_a), f(g.br_angmin), f(g.br_angmax)
        d.gen_bus = i(g.gen_bus)
        d.pmin, d.pmax, d.qmin, d.qmax = f(g.gen_pmin), f(g.gen_pmax), f(g.gen_qmin), f(g.gen_qmax)
        d.c2, d.c1, d.c0 = f(g.gen_c2), f(g.gen_c1), f(g.gen_c0)
        d.load_bus = i(g.load_bus)
        d.pd, d.qd = f(g.load_pd), f(g.load_qd)
        d.ramp_ratio = float(g.ramp_ratio)

    def _fill_storage(self, d, st):
        if st is None:
            d.nstor, d.dt = 0, 1.0
            return
        keep = self._keep

        def f(a):
            a = _f64(a)
            keep.append(a)
            return _p(a, _f64p)

        b = _i32(st.bus)
        keep.append(b)
        d.nstor, d.bus, d.dt = st.nstor, _p(b, _i32p), float(st.dt)
        for name in ("energy_rating", "charge_rating", "discharge_rating", "thermal_rating", "eta_c", "eta_d",
                     "r", "p_loss", "qmin", "qmax", "e_init"):
            setattr(d, name, f(getattr(st, name)))

    def __del__(self):
        if getattr(self, "ctx", None) and _lib is not None:
            _lib.ora_destroy(self.ctx)
            self.ctx = None

    def jac_pattern(self):
        r = np.empty(self.nnzj, np.int64)
        c = np.empty(self.nnzj, np.int64)
        lib().ora_jac_pattern(self.ctx, _p(r, _i64p), _p(c, _i64p))
        return r, c

    def hess_pattern(self):
        r = np.empty(self.nnzh, np.int64)
        c = np.empty(self.nnzh, np.int64)
        lib().ora_hess_pattern(self.ctx, _p(r, _i64p), _p(c, _i64p))
        return r, c

    def bounds(self):
        xl, xu = np.empty(self.n), np.empty(self.n)
        gl, gu = np.empty(self.m), np.empty(self.m)
        lib().ora_bounds(self.ctx, _p(xl, _f64p), _p(xu, _f64p), _p(gl, _f64p), _p(gu, _f64p))
        return xl, xu, gl, gu

    def obj(self, x, with_scale: bool = False):
        """f(x); with_scale: (f, the sum of the magnitudes of its terms)."""
        x = _f64(x)
        f = lib().ora_obj(self.ctx, _p(x, _f64p))
        return (f, lib().ora_obj_scale(self.ctx, _p(x, _f64p))) if with_scale else f

    def grad(self, x):
        x = _f64(x)
        g = np.empty(self.n)
        lib().ora_grad(self.ctx, _p(x, _f64p), _p(g, _f64p))
        return g

    def cons(self, x, with_scale: bool = False):
        x = _f64(x)
        c = np.empty(self.m)
        s = np.empty(self.m) if with_scale else None
        lib().ora_cons(self.ctx, _p(x, _f64p), _p(c, _f64p), _p(s, _f64p))
        return (c, s) if with_scale else c

    def jac(self, x, with_scale: bool = False):
        x = _f64(x)
        v = np.empty(self.nnzj)
        s = np.empty(self.nnzj) if with_scale else None
        if lib().ora_jac(self.ctx, _p(x, _f64p), _p(v, _f64p), _p(s, _f64p)):
            raise RuntimeError("oracle jac: " + lib().ora_error().decode())
        return (v, s) if with_scale else v

    def hess(self, x, lam, sigma: float = 1.0, with_scale: bool = False):
        x, lam = _f64(x), _f64(lam)
        v = np.empty(self.nnzh)
        s = np.empty(self.nnzh) if with_scale else None
        if lib().ora_hess(self.ctx, _p(x, _f64p), _p(lam, _f64p), float(sigma), _p(v, _f64p),
                          _p(s, _f64p)):
            raise RuntimeError("oracle hess: " + lib().ora_error().decode())
        return (v, s) if with_scale else v

    def cvio(self, x):
        x = _f64(x)
        cv, vv = ctypes.c_double(), ctypes.c_double()
        lib().ora_cvio(self.ctx, _p(x, _f64p), ctypes.byref(cv), ctypes.byref(vv))
        return cv.value, vv.value
