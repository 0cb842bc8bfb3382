"""Python binding of libopf (include/opf.h): argument marshalling only.

Every evaluation runs in the library's CUDA kernels. If libopf.so is missing
the import fails loudly; there is no CPU path.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libopf.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "opf.h")

OPF_OK, OPF_EINVAL, OPF_ENOMEM, OPF_ECUDA, OPF_ESTATE = 0, 1, 2, 3, 4
OPF_JAC, OPF_HESS = 0, 1
OPF_PHASE_BRANCH, OPF_PHASE_BUS = 1, 2

_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_vp = ctypes.c_void_p


class OpfNetwork(ctypes.Structure):
    _fields_ = [
        ("nbus", ctypes.c_int32), ("nbranch", ctypes.c_int32), ("ngen", ctypes.c_int32),
        ("nload", ctypes.c_int32), ("nperiod", ctypes.c_int32), ("ref_bus", ctypes.c_int32),
        ("bus_vmin", _f64p), ("bus_vmax", _f64p), ("bus_gs", _f64p), ("bus_bs", _f64p),
        ("br_f", _i32p), ("br_t", _i32p), ("br_r", _f64p), ("br_x", _f64p), ("br_b", _f64p),
        ("br_tap", _f64p), ("br_shift", _f64p), ("br_rate_a", _f64p), ("br_angmin", _f64p),
        ("br_angmax", _f64p), ("gen_bus", _i32p), ("gen_pmin", _f64p), ("gen_pmax", _f64p),
        ("gen_qmin", _f64p), ("gen_qmax", _f64p), ("gen_c2", _f64p), ("gen_c1", _f64p),
        ("gen_c0", _f64p), ("load_bus", _i32p), ("load_pd", _f64p), ("load_qd", _f64p),
        ("ramp_ratio", ctypes.c_double),
    ]


class OpfStorage(ctypes.Structure):
    _fields_ = [("nstor", ctypes.c_int32), ("bus", _i32p),
                ("energy_rating", _f64p), ("charge_rating", _f64p), ("discharge_rating", _f64p),
                ("thermal_rating", _f64p), ("eta_c", _f64p), ("eta_d", _f64p), ("r", _f64p),
                ("p_loss", _f64p), ("qmin", _f64p), ("qmax", _f64p), ("e_init", _f64p),
                ("dt", ctypes.c_double)]


class OpfBatchOpts(ctypes.Structure):
    _fields_ = [("link_ratio", ctypes.c_double), ("link_ratios", ctypes.POINTER(ctypes.c_double)),
                ("reserve", ctypes.c_double), ("form", ctypes.c_int32),
                ("storage", ctypes.POINTER(OpfStorage)), ("storage_complementarity", ctypes.c_int32)]


FORMS = {"polar": 0, "rect": 1}


class OpfLaunch(ctypes.Structure):
    _fields_ = [("branch_block", ctypes.c_int32), ("bus_block", ctypes.c_int32),
                ("branch_ctas_per_sm", ctypes.c_int32), ("bus_ctas_per_sm", ctypes.c_int32),
                ("bus_order", ctypes.c_int32), ("branch_occupancy", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class OpfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libopf error {code}: {msg}")
        self.code = code


_lib = None


def lib():
    """Load libopf.so (built by paper_2510_12897_b300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_2510_12897_b300.build` (there is no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    netp = ctypes.POINTER(OpfNetwork)
    mp = ctypes.POINTER(_vp)
    sig = {
        "opf_model_create": [netp, mp],
        "opf_batch_create": [netp, ctypes.c_int32, ctypes.POINTER(OpfBatchOpts), mp],
        "opf_structure_create": [netp, ctypes.c_int32, ctypes.POINTER(OpfBatchOpts), mp],
        "opf_model_destroy": [_vp],
        "opf_dims": [_vp, _i64p, _i64p, _i64p, _i64p],
        "opf_sparsity": [_vp, ctypes.c_int32, _i64p, _i64p],
        "opf_bounds": [_vp, _f64p, _f64p, _f64p, _f64p],
        "opf_eval_obj_grad": [_vp, _vp, _vp, _vp, _vp],
        "opf_eval_cons": [_vp, _vp, _vp, _vp],
        "opf_eval_jac": [_vp, _vp, _vp, _vp],
        "opf_eval_hess": [_vp, _vp, _vp, ctypes.c_double, _vp, _vp],
        "opf_eval_jac_hess": [_vp, _vp, _vp, ctypes.c_double, _vp, _vp, _vp],
        "opf_eval_all": [_vp, _vp, _vp, ctypes.c_double, _vp, _vp, _vp, _vp, _vp, _vp],
        "opf_eval_phases": [_vp, ctypes.c_int32, _vp, _vp, ctypes.c_double, _vp, _vp, _vp, _vp, _vp,
                            _vp],
        "opf_eval_all_noalloc": [_vp, _vp, _vp, ctypes.c_double, _vp, _vp, _vp, _vp, _vp, _vp],
        "opf_eval_all_host": [_vp, _vp, _vp, ctypes.c_double, _vp, _vp, _vp, _vp, _vp, _vp],
        "opf_eval_all_host_async": [_vp, _vp, _vp, ctypes.c_double, _vp, _vp, _vp, _vp, _vp, _vp],
        "opf_flat_start": [_vp, _vp, _vp],
        "opf_sincos": [_vp, _vp, ctypes.c_int64, _vp, _vp, _vp],
        "opf_eval_jtprod": [_vp, _vp, _vp, _vp, _vp],
        "opf_eval_flows": [_vp, _vp, _vp],
        "opf_set_loads": [_vp, _vp, _vp, _vp],
        "opf_get_launch": [_vp, ctypes.POINTER(OpfLaunch)],
        "opf_set_launch": [_vp, ctypes.POINTER(OpfLaunch)],
        "opf_autotune": [_vp, _vp, _vp, ctypes.c_int32, _vp, ctypes.POINTER(OpfLaunch), _f64p],
        "opf_autotune_list": [_vp, _vp, _vp, ctypes.c_int32, _vp, ctypes.POINTER(OpfLaunch), _f64p, ctypes.c_int32,
                              ctypes.POINTER(ctypes.c_int32)],
        "opf_host_register": [_vp, ctypes.c_size_t],
        "opf_host_unregister": [_vp],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L.opf_last_error.restype = ctypes.c_char_p
    L.opf_last_error.argtypes = []
    _lib = L
    return L


def host_register(array) -> None:
    """Page-lock a host numpy array (or CPU tensor) for this library's copies."""
    ptr, nbytes = _host_buf(array)
    _check(lib().opf_host_register(ptr, nbytes))


def host_unregister(array) -> None:
    _check(lib().opf_host_unregister(_host_buf(array)[0]))


def _host_buf(a):
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("host buffer must be contiguous")
        return a.ctypes.data, a.nbytes
    if not a.is_contiguous() or a.is_cuda:
        raise ValueError("host buffer must be a contiguous CPU tensor")
    return a.data_ptr(), a.numel() * a.element_size()


def declared_symbols(header: str = HEADER) -> list[str]:
    """Entry points declared in include/opf.h."""
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(opf_[a-z_]+)\s*\(", text)))


def _check(rc):
    if rc != OPF_OK:
        raise OpfError(rc, lib().opf_last_error().decode())


def _net_struct(g, keep):
    def f(a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        keep.append(a)
        return a.ctypes.data_as(_f64p)

    def i(a):
        a = np.ascontiguousarray(a, dtype=np.int32)
        keep.append(a)
        return a.ctypes.data_as(_i32p)

    d = OpfNetwork()
    d.nbus, d.nbranch, d.ngen = g.nbus, len(g.br_f), len(g.gen_bus)
    d.nload, d.nperiod, d.ref_bus = len(g.load_bus), int(g.load_pd.shape[0]), int(g.ref_bus)
    d.bus_vmin, d.bus_vmax, d.bus_gs, d.bus_bs = f(g.bus_vmin), f(g.bus_vmax), f(g.bus_gs), f(g.bus_bs)
    d.br_f, d.br_t = i(g.br_f), i(g.br_t)
    d.br_r, d.br_x, d.br_b = f(g.br_r), f(g.br_x), f(g.br_b)
    d.br_tap, d.br_shift = f(g.br_tap), f(g.br_shift)
    d.br_rate_a, d.br_angmin, d.br_angmax = f(g.br_rate_a), f(g.br_angmin), f(g.br_angmax)
    d.gen_bus = i(g.gen_bus)
    d.gen_pmin, d.gen_pmax = f(g.gen_pmin), f(g.gen_pmax)
    d.gen_qmin, d.gen_qmax = f(g.gen_qmin), f(g.gen_qmax)
    d.gen_c2, d.gen_c1, d.gen_c0 = f(g.gen_c2), f(g.gen_c1), f(g.gen_c0)
    d.load_bus = i(g.load_bus)
    d.load_pd, d.load_qd = f(g.load_pd), f(g.load_qd)
    d.ramp_ratio = float(g.ramp_ratio)
    return d


def _storage_struct(st, keep):
    d = OpfStorage()
    if st is None:
        d.nstor, d.dt = 0, 1.0
        return d

    def f(a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        keep.append(a)
        return a.ctypes.data_as(_f64p)

    b = np.ascontiguousarray(st.bus, dtype=np.int32)
    keep.append(b)
    d.nstor, d.bus, d.dt = st.nstor, b.ctypes.data_as(_i32p), float(st.dt)
    for name in ("energy_rating", "charge_rating", "discharge_rating", "thermal_rating", "eta_c", "eta_d", "r",
                 "p_loss", "qmin", "qmax", "e_init"):
        setattr(d, name, f(getattr(st, name)))
    return d


def _ptr(t, n=None, name="buffer"):
    """Device pointer of a contiguous float64 CUDA tensor (or None)."""
    if t is None:
        return None
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    if n is not None and t.numel() < n:
        raise ValueError(f"{name} has {t.numel()} entries, needs {n}")
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


class Model:
    """A GPU model of one grid, a multi-period grid or a batch of grids.

    ``grids`` is one ``synth.Grid``-like object (attributes as in opf.h) or a
    list of them (a batch). ``structure_only=True`` builds the host layout
    only (dims, patterns, bounds) without touching a GPU. ``form`` is
    "polar" (va, vm) or "rect" (vr, vi). Grids carrying ``storage`` (a
    ``synth.Storage``) get the storage variables and rows; ``compl`` adds
    the complementarity rows.
    """

    def __init__(self, grids, link_ratio: float = 0.0, structure_only: bool = False, link_ratios=None,
                 reserve: float = 0.0, form: str = "polar", compl: bool = False):
        if form not in FORMS:
            raise ValueError("form must be 'polar' or 'rect'")
        self.form = form
        batch = (isinstance(grids, (list, tuple)) or link_ratios is not None or reserve > 0.0
                 or form != "polar" or compl
                 or any(getattr(g, "storage", None) is not None
                        for g in (grids if isinstance(grids, (list, tuple)) else [grids])))
        gl = list(grids) if isinstance(grids, (list, tuple)) else [grids]
        self._keep = []
        arr = (OpfNetwork * len(gl))(*[_net_struct(g, self._keep) for g in gl])
        h = _vp()
        L = lib()
        lr = None
        if link_ratios is not None:
            lr = np.ascontiguousarray(link_ratios, dtype=np.float64)
            self._keep.append(lr)
        stor = None
        if any(getattr(g, "storage", None) is not None for g in gl):
            stor = (OpfStorage * len(gl))(*[_storage_struct(getattr(g, "storage", None), self._keep) for g in gl])
        opts = OpfBatchOpts(float(link_ratio), None if lr is None else lr.ctypes.data_as(_f64p), float(reserve),
                            FORMS[form], stor, 1 if compl else 0)
        if structure_only:
            _check(L.opf_structure_create(arr, len(gl), ctypes.byref(opts), ctypes.byref(h)))
        elif batch:
            _check(L.opf_batch_create(arr, len(gl), ctypes.byref(opts), ctypes.byref(h)))
        else:
            _check(L.opf_model_create(arr, ctypes.byref(h)))
        self.h = h
        self._keep = None  # the library copied everything
        n, m, nj, nh = (ctypes.c_int64() for _ in range(4))
        _check(L.opf_dims(h, ctypes.byref(n), ctypes.byref(m), ctypes.byref(nj), ctypes.byref(nh)))
        self.n, self.m, self.nnzj, self.nnzh = n.value, m.value, nj.value, nh.value

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            lib().opf_model_destroy(self.h)
            self.h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ host --
    def sparsity(self, kind: int):
        nnz = self.nnzj if kind == OPF_JAC else self.nnzh
        r = np.empty(nnz, np.int64)
        c = np.empty(nnz, np.int64)
        _check(lib().opf_sparsity(self.h, kind, r.ctypes.data_as(_i64p), c.ctypes.data_as(_i64p)))
        return r, c

    def jac_pattern(self):
        return self.sparsity(OPF_JAC)

    def hess_pattern(self):
        return self.sparsity(OPF_HESS)

    def bounds(self):
        xl, xu = np.empty(self.n), np.empty(self.n)
        gl, gu = np.empty(self.m), np.empty(self.m)
        _check(lib().opf_bounds(self.h, *(a.ctypes.data_as(_f64p) for a in (xl, xu, gl, gu))))
        return xl, xu, gl, gu

    # ------------------------------------------------------------ device --
    def eval_obj_grad(self, x, obj=None, grad=None, stream=None):
        _check(lib().opf_eval_obj_grad(self.h, _ptr(x, self.n, "x"), _ptr(obj, 1, "obj"),
                                       _ptr(grad, self.n, "grad"), _stream(stream)))

    def eval_cons(self, x, c, stream=None):
        _check(lib().opf_eval_cons(self.h, _ptr(x, self.n, "x"), _ptr(c, self.m, "c"), _stream(stream)))

    def eval_jac(self, x, jv, stream=None):
        _check(lib().opf_eval_jac(self.h, _ptr(x, self.n, "x"), _ptr(jv, self.nnzj, "jvals"),
                                  _stream(stream)))

    def eval_hess(self, x, lam, sigma, hv, stream=None):
        _check(lib().opf_eval_hess(self.h, _ptr(x, self.n, "x"), _ptr(lam, self.m, "lambda"),
                                   float(sigma), _ptr(hv, self.nnzh, "hvals"), _stream(stream)))

    def eval_jac_hess(self, x, lam, sigma, jv, hv, stream=None):
        _check(lib().opf_eval_jac_hess(self.h, _ptr(x, self.n, "x"), _ptr(lam, self.m, "lambda"),
                                       float(sigma), _ptr(jv, self.nnzj, "jvals"),
                                       _ptr(hv, self.nnzh, "hvals"), _stream(stream)))

    def eval_all(self, x, lam=None, sigma=1.0, obj=None, grad=None, c=None, jv=None, hv=None,
                 stream=None):
        _check(lib().opf_eval_all(self.h, _ptr(x, self.n, "x"), _ptr(lam, self.m, "lambda"),
                                  float(sigma), _ptr(obj, 1, "obj"), _ptr(grad, self.n, "grad"),
                                  _ptr(c, self.m, "c"), _ptr(jv, self.nnzj, "jvals"),
                                  _ptr(hv, self.nnzh, "hvals"), _stream(stream)))

    def eval_all_noalloc(self, x, lam=None, sigma=1.0, obj=None, grad=None, c=None, jv=None,
                         hv=None, stream=None):
        """eval_all with the library's static scratch: no allocation in the
        call (see opf_eval_all_noalloc in include/opf.h for the limits)."""
        _check(lib().opf_eval_all_noalloc(self.h, _ptr(x, self.n, "x"), _ptr(lam, self.m, "lambda"),
                                          float(sigma), _ptr(obj, 1, "obj"), _ptr(grad, self.n, "grad"),
                                          _ptr(c, self.m, "c"), _ptr(jv, self.nnzj, "jvals"),
                                          _ptr(hv, self.nnzh, "hvals"), _stream(stream)))

    def eval_phases(self, phases, x, lam=None, sigma=1.0, obj=None, grad=None, c=None, jv=None,
                    hv=None, stream=None):
        _check(lib().opf_eval_phases(self.h, int(phases), _ptr(x, self.n, "x"),
                                     _ptr(lam, self.m, "lambda"), float(sigma), _ptr(obj, 1, "obj"),
                                     _ptr(grad, self.n, "grad"), _ptr(c, self.m, "c"),
                                     _ptr(jv, self.nnzj, "jvals"), _ptr(hv, self.nnzh, "hvals"),
                                     _stream(stream)))

    def eval_all_host(self, x, lam=None, sigma=1.0, obj=None, grad=None, c=None, jv=None, hv=None,
                      stream=None, pipelined=False):
        """Host arrays (numpy or CPU tensors, float64, contiguous; memory
        page-locked with host_register copies at full speed) in and out.
        Synchronises, unless `pipelined`: then the call returns at once, its
        copies and evaluation overlap those of the next call, and the host
        outputs are complete when `stream` has been synchronised."""
        def hp(a, n, name):
            if a is None:
                return None
            if hasattr(a, "data_ptr"):
                if a.is_cuda or a.dtype.itemsize != 8 or not a.is_contiguous() or a.numel() < n:
                    raise TypeError(f"{name}: contiguous float64 host tensor of {n} entries expected")
                return a.data_ptr()
            if a.dtype != np.float64 or not a.flags.c_contiguous or a.size < n:
                raise TypeError(f"{name}: contiguous float64 array of {n} entries expected")
            return a.ctypes.data
        fn = lib().opf_eval_all_host_async if pipelined else lib().opf_eval_all_host
        _check(fn(self.h, hp(x, self.n, "x"), hp(lam, self.m, "lambda"), float(sigma), hp(obj, 1, "obj"),
                  hp(grad, self.n, "grad"), hp(c, self.m, "c"), hp(jv, self.nnzj, "jvals"),
                  hp(hv, self.nnzh, "hvals"), _stream(stream)))

    def flat_start(self, x, stream=None):
        _check(lib().opf_flat_start(self.h, _ptr(x, self.n, "x"), _stream(stream)))

    def eval_jtprod(self, x, v, out, stream=None):
        _check(lib().opf_eval_jtprod(self.h, _ptr(x, self.n, "x"), _ptr(v, self.m, "v"),
                                     _ptr(out, self.n, "out"), _stream(stream)))

    def eval_flows(self, x, stream=None):
        _check(lib().opf_eval_flows(self.h, _ptr(x, self.n, "x"), _stream(stream)))

    def set_loads(self, pd, qd, stream=None):
        """pd, qd: float64 CUDA tensors holding every instance's [nperiod][nload]
        loads, instances concatenated."""
        _check(lib().opf_set_loads(self.h, _ptr(pd, None, "pd"), _ptr(qd, None, "qd"), _stream(stream)))

    def sincos(self, d, sn, cs, stream=None):
        n = d.numel()
        _check(lib().opf_sincos(self.h, _ptr(d, n, "angles"), n, _ptr(sn, n, "sin"), _ptr(cs, n, "cos"),
                                _stream(stream)))

    def get_launch(self) -> dict:
        cfg = OpfLaunch()
        _check(lib().opf_get_launch(self.h, ctypes.byref(cfg)))
        return cfg.as_dict()

    def set_launch(self, branch_block=128, bus_block=128, branch_ctas_per_sm=0, bus_ctas_per_sm=0,
                   bus_order=0, branch_occupancy=0):
        cfg = OpfLaunch(branch_block, bus_block, branch_ctas_per_sm, bus_ctas_per_sm, bus_order,
                        branch_occupancy)
        _check(lib().opf_set_launch(self.h, ctypes.byref(cfg)))

    def autotune(self, x, lam, reps: int = 20, stream=None):
        cfg = OpfLaunch()
        us = ctypes.c_double()
        _check(lib().opf_autotune(self.h, _ptr(x, self.n, "x"), _ptr(lam, self.m, "lambda"), int(reps),
                                  _stream(stream), ctypes.byref(cfg), ctypes.byref(us)))
        return cfg.as_dict(), us.value

    def autotune_list(self, x, lam, reps: int = 20, max_shapes: int = 8, stream=None):
        """The autotuner's finalists, fastest first: [(shape dict, us per eval)]."""
        shapes = (OpfLaunch * int(max_shapes))()
        us = (ctypes.c_double * int(max_shapes))()
        k = ctypes.c_int32()
        _check(lib().opf_autotune_list(self.h, _ptr(x, self.n, "x"), _ptr(lam, self.m, "lambda"), int(reps),
                                       _stream(stream), shapes, us, int(max_shapes), ctypes.byref(k)))
        return [(shapes[q].as_dict(), us[q]) for q in range(k.value)]
