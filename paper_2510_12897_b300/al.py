"""Python binding of the augmented-Lagrangian loop (include/opf_al.h). Every
step runs in libopf's kernels; this module passes device pointers."""
from __future__ import annotations

import ctypes

from . import opf

_vp = ctypes.c_void_p


class AlOpts(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_double), ("lr", ctypes.c_double)]


_ready = False


def _lib():
    global _ready
    L = opf.lib()
    if not _ready:
        sig = {
            "opf_al_create": [_vp, ctypes.POINTER(AlOpts), ctypes.POINTER(_vp)],
            "opf_al_destroy": [_vp],
            "opf_al_iterate": [_vp, _vp, _vp, ctypes.c_int32, _vp, _vp],
            "opf_al_update": [_vp, _vp, _vp, _vp, _vp],
            "opf_al_reset": [_vp, ctypes.c_double, ctypes.c_double],
            "opf_al_newton": [_vp, _vp, _vp, ctypes.c_int32, _vp, _vp, _vp],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        _ready = True
    return L


class AugLag:
    """Adam inner iterations and multiplier updates on one model."""

    def __init__(self, model: opf.Model, rho: float = 10.0, lr: float = 1e-3):
        h = _vp()
        opf._check(_lib().opf_al_create(model.h, ctypes.byref(AlOpts(rho, lr)), ctypes.byref(h)))
        self.h, self.model = h, model

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            _lib().opf_al_destroy(self.h)
            self.h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def iterate(self, x, lam, iters: int, stats=None, stream=None):
        M = self.model
        opf._check(_lib().opf_al_iterate(self.h, opf._ptr(x, M.n, "x"), opf._ptr(lam, M.m, "lambda"), int(iters),
                                         opf._ptr(stats, 3, "stats"), opf._stream(stream)))

    def update(self, x, lam, stats=None, stream=None):
        M = self.model
        opf._check(_lib().opf_al_update(self.h, opf._ptr(x, M.n, "x"), opf._ptr(lam, M.m, "lambda"),
                                        opf._ptr(stats, 3, "stats"), opf._stream(stream)))

    def newton(self, x, lam, cg_iters: int = 50, stats=None, step=None, stream=None):
        """One projected Newton-CG step on x (see opf_al_newton)."""
        M = self.model
        opf._check(_lib().opf_al_newton(self.h, opf._ptr(x, M.n, "x"), opf._ptr(lam, M.m, "lambda"), int(cg_iters),
                                        opf._ptr(stats, 3, "stats"), opf._ptr(step, M.n, "step"),
                                        opf._stream(stream)))

    def reset(self, rho: float, lr: float):
        opf._check(_lib().opf_al_reset(self.h, float(rho), float(lr)))
