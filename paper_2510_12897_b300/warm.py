"""Python binding of the learned warm start (include/opf_warm.h) and a
training driver. Every step runs in libopf's kernels; this module only
passes device pointers and loops over batches."""
from __future__ import annotations

import ctypes
import time

import numpy as np

from . import opf

_vp = ctypes.c_void_p


class WarmOpts(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int32), ("hidden", ctypes.c_int32), ("penalty", ctypes.c_double),
                ("lr", ctypes.c_double), ("lr_out", ctypes.c_double), ("va_scale", ctypes.c_double),
                ("seed", ctypes.c_uint64)]


_ready = False


def _lib():
    global _ready
    L = opf.lib()
    if not _ready:
        sig = {
            "opf_warm_create": [ctypes.POINTER(opf.OpfNetwork), ctypes.POINTER(WarmOpts), ctypes.POINTER(_vp)],
            "opf_warm_destroy": [_vp],
            "opf_warm_dims": [_vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                              ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)],
            "opf_warm_train_step": [_vp, _vp, _vp, _vp, _vp],
            "opf_warm_predict": [_vp, _vp, _vp, _vp, _vp],
            "opf_warm_forward": [_vp, _vp, _vp, _vp, _vp],
            "opf_warm_backward": [_vp, _vp, _vp, _vp],
            "opf_warm_loss_grad": [_vp, _vp, _vp, _vp, _vp, _vp, _vp],
            "opf_warm_set_lr": [_vp, ctypes.c_double, ctypes.c_double],
            "opf_warm_get_params": [_vp, _vp],
            "opf_warm_get_activations": [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
            "opf_warm_set_params": [_vp, _vp],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        _ready = True
    return L


def _p(t, n, name, dtype):
    import torch
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous {dtype} CUDA tensor")
    if t.numel() < n:
        raise ValueError(f"{name} has {t.numel()} entries, needs {n}")
    return t.data_ptr()


class WarmStart:
    """The warm-start network of one single-period grid."""

    def __init__(self, grid, batch=4096, hidden=1024, penalty=1e3, lr=1e-4, lr_out=1e-2, va_scale=1.0,
                 seed=0):
        keep = []
        net = opf._net_struct(grid, keep)
        opts = WarmOpts(batch, hidden, penalty, lr, lr_out, va_scale, seed)
        h = _vp()
        opf._check(_lib().opf_warm_create(ctypes.byref(net), ctypes.byref(opts), ctypes.byref(h)))
        self.h = h
        self.grid = grid
        self.batch = batch
        a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        d = ctypes.c_int64()
        opf._check(_lib().opf_warm_dims(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)))
        self.n_in, self.n_out, self.n_x, self.n_params = a.value, b.value, c.value, d.value
        self.nload = grid.nload

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            _lib().opf_warm_destroy(self.h)
            self.h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _loads(self, pd, qd):
        import torch
        n = self.batch * self.nload
        return _p(pd, n, "pd", torch.float64), _p(qd, n, "qd", torch.float64)

    def train_step(self, pd, qd, stats=None, stream=None):
        import torch
        a, b = self._loads(pd, qd)
        opf._check(_lib().opf_warm_train_step(self.h, a, b, _p(stats, 3, "stats", torch.float64),
                                              opf._stream(stream)))

    def predict(self, pd, qd, x, stream=None):
        import torch
        a, b = self._loads(pd, qd)
        opf._check(_lib().opf_warm_predict(self.h, a, b, _p(x, self.n_x * self.batch, "x", torch.float64),
                                           opf._stream(stream)))

    def forward(self, pd, qd, y, stream=None):
        import torch
        a, b = self._loads(pd, qd)
        opf._check(_lib().opf_warm_forward(self.h, a, b, _p(y, self.batch * self.n_out, "y", torch.float32),
                                           opf._stream(stream)))

    def backward(self, dy, grad, stream=None):
        import torch
        opf._check(_lib().opf_warm_backward(self.h, _p(dy, self.batch * self.n_out, "dy", torch.float32),
                                            _p(grad, self.n_params, "grad", torch.float32),
                                            opf._stream(stream)))

    def loss_grad(self, pd, qd, y, dy, stats=None, stream=None):
        import torch
        a, b = self._loads(pd, qd)
        opf._check(_lib().opf_warm_loss_grad(self.h, a, b, _p(y, self.batch * self.n_out, "y", torch.float32),
                                             _p(dy, self.batch * self.n_out, "dy", torch.float32),
                                             _p(stats, 3, "stats", torch.float64), opf._stream(stream)))

    def set_lr(self, lr, lr_out):
        opf._check(_lib().opf_warm_set_lr(self.h, float(lr), float(lr_out)))

    def get_params(self):
        out = np.empty(self.n_params, np.float32)
        opf._check(_lib().opf_warm_get_params(self.h, out.ctypes.data))
        return out

    def activations(self):
        """(u, z1, h1, z2, h2, dz2, dz1) of the last forward/backward pass as
        float64 arrays (BF16 ones widened exactly); see
        opf_warm_get_activations."""
        hid = _hidden_of(self.n_params, self.n_in, self.n_out)
        B = self.batch
        u = np.empty((B, self.n_in), np.uint16)
        h1, h2 = np.empty((B, hid), np.uint16), np.empty((B, hid), np.uint16)
        z1, z2, dz2, dz1 = (np.empty((B, hid), np.float32) for _ in range(4))
        opf._check(_lib().opf_warm_get_activations(self.h, *(a.ctypes.data for a in (u, z1, h1, z2, h2, dz2, dz1))))

        def widen(a):  # BF16 words are the top halves of FP32 words
            return (a.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
        return (widen(u), z1.astype(np.float64), widen(h1), z2.astype(np.float64), widen(h2),
                dz2.astype(np.float64), dz1.astype(np.float64))

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        if p.size != self.n_params:
            raise ValueError("wrong parameter count")
        opf._check(_lib().opf_warm_set_params(self.h, p.ctypes.data))

    def param_views(self, flat):
        """W1, b1, W2, b2, W3, b3 views of a flat parameter array."""
        Kin, Nout = self.n_in, self.n_out
        hid = _hidden_of(self.n_params, self.n_in, self.n_out)
        o = 0
        out = []
        for shape in ((hid, Kin), (hid,), (hid, hid), (hid,), (Nout, hid), (Nout,)):
            k = int(np.prod(shape))
            out.append(flat[o:o + k].reshape(shape))
            o += k
        return out


def _hidden_of(n_params, n_in, n_out):
    # n_params = H n_in + H + H^2 + H + n_out H + n_out
    a, b, c = 1.0, n_in + 2 + n_out, n_out - n_params
    return int(round((-b + (b * b - 4 * a * c) ** 0.5) / (2 * a)))


def train(ws: WarmStart, pd_all, qd_all, epochs: int, lr: float = 1e-4, lr_out: float = 1e-2,
          decay: float = 100.0, stream=None, log=None):
    """Adam over shuffled batches of the sample tensors (float64 CUDA,
    [count][nload]); both learning rates decay on a cosine from their
    starting values to 1/decay of them. Returns the per-epoch mean
    statistics (loss, cost, sum of squared residuals)."""
    import torch
    dev = pd_all.device
    count = pd_all.shape[0]
    nb = count // ws.batch
    stats = torch.zeros((nb, 3), dtype=torch.float64, device=dev)
    g = torch.Generator(device="cpu")
    g.manual_seed(1234)
    history = []
    total = epochs * nb
    step = 0
    t0 = time.perf_counter()
    for ep in range(epochs):
        perm = torch.randperm(count, generator=g)[: nb * ws.batch].to(dev)
        pd_e = pd_all[perm].contiguous()
        qd_e = qd_all[perm].contiguous()
        for b in range(nb):
            frac = step / max(1, total - 1)
            scale = 1.0 / decay + 0.5 * (1.0 - 1.0 / decay) * (1 + np.cos(np.pi * frac))
            ws.set_lr(lr * scale, lr_out * scale)
            sl = slice(b * ws.batch, (b + 1) * ws.batch)
            ws.train_step(pd_e[sl], qd_e[sl], stats[b], stream=stream)
            step += 1
        m = stats.mean(0).cpu().numpy()
        history.append(m)
        if log:
            log(f"epoch {ep}: loss {m[0]:.4g} cost {m[1]:.4g} res2 {m[2]:.4g} "
                f"({time.perf_counter() - t0:.1f} s)")
    return np.array(history)
