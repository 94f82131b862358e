"""Python binding of the surface surrogate (include/tsurr.h, inside libtsim.so).

Argument marshalling only: forward, backward and Adam run in the library's
tensor-core kernels.  Arrays are numpy (host, ``on_device=0``) or contiguous
torch CUDA tensors (``on_device=1``); a non-zero status raises ``TsimError``.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import inputs as _inputs
from . import tsim as _t

TSURR_CIN = 12
TSURR_COUT = 4

EXPORTS = ["tsurr_create", "tsurr_num_params", "tsurr_set_params", "tsurr_get_params", "tsurr_get_grads",
           "tsurr_forward", "tsurr_backward", "tsurr_adam", "tsurr_sync", "tsurr_destroy", "tsurr_features",
           "tsurr_indicator"]

# (cin, cout, stride, upsample, relu, skip source layer or -1) per layer; the
# network input is padded from 12 to 16 channels, the output stored as 16.
LAYERS = [(16, 32, 1, 0, 1, -1), (32, 64, 2, 0, 1, -1), (64, 128, 2, 0, 1, -1), (128, 256, 2, 0, 1, -1),
          (256, 256, 1, 0, 1, -1), (256, 128, 1, 1, 1, 2), (128, 64, 1, 1, 1, 1), (64, 32, 1, 1, 1, 0),
          (32, 16, 1, 0, 0, -1)]

_sig_done = False


def load():
    global _sig_done
    L = _t.load()
    if not _sig_done:
        P, vp = C.POINTER, C.c_void_p
        sig = {
            "tsurr_create": (C.c_int, [C.c_int, C.c_int, C.c_int, vp, P(vp)]),
            "tsurr_num_params": (C.c_int64, [vp]),
            "tsurr_set_params": (C.c_int, [vp, vp, C.c_int64, C.c_int]),
            "tsurr_get_params": (C.c_int, [vp, vp, C.c_int64, C.c_int]),
            "tsurr_get_grads": (C.c_int, [vp, vp, C.c_int64, C.c_int]),
            "tsurr_forward": (C.c_int, [vp, vp, C.c_int, vp, C.c_int]),
            "tsurr_backward": (C.c_int, [vp, vp, vp, vp, C.c_int, P(C.c_double), C.c_int]),
            "tsurr_adam": (C.c_int, [vp, C.c_float, C.c_float, C.c_float, C.c_float, C.c_int]),
            "tsurr_sync": (C.c_int, [vp]),
            "tsurr_destroy": (None, [vp]),
            "tsurr_features": (C.c_int, [vp, vp, C.c_int, C.c_int, C.c_int, vp, vp]),
            "tsurr_indicator": (C.c_int, [vp, vp, C.c_int, C.c_int, C.c_int, vp, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _sig_done = True
    return L


def param_layout():
    """[(w_offset, w_shape, b_offset, b_len)] for the flat FP32 parameter vector."""
    out, off = [], 0
    for cin, cout, *_ in LAYERS:
        shape = (cout, 3, 3, cin)
        nw = cout * 9 * cin
        out.append((off, shape, off + nw, cout))
        off += nw + cout
    return out


def num_params() -> int:
    lay = param_layout()
    return lay[-1][2] + lay[-1][3]


def init_params(seed: int) -> np.ndarray:
    """He-normal initial weights, zero biases (seeded)."""
    return _inputs.surrogate_params(seed)


def tsurr_create(max_batch, height, width, stream=None):
    h = C.c_void_p()
    _t._check(load().tsurr_create(int(max_batch), int(height), int(width), _t._stream_handle(stream), C.byref(h)))
    return h


def tsurr_num_params(net) -> int:
    return int(load().tsurr_num_params(net))


def tsurr_set_params(net, p):
    ptr, on, keep = _t._ptr(p, np.float32)
    n = keep.numel() if hasattr(keep, "numel") else keep.size
    _t._check(load().tsurr_set_params(net, ptr, int(n), on))


def tsurr_get_params(net, out=None):
    arr = np.empty(tsurr_num_params(net), np.float32) if out is None else out
    ptr, on, _ = _t._ptr(arr, np.float32)
    _t._check(load().tsurr_get_params(net, ptr, tsurr_num_params(net), on))
    return arr


def tsurr_get_grads(net, out=None):
    arr = np.empty(tsurr_num_params(net), np.float32) if out is None else out
    ptr, on, _ = _t._ptr(arr, np.float32)
    _t._check(load().tsurr_get_grads(net, ptr, tsurr_num_params(net), on))
    return arr


def tsurr_forward(net, x, out=None):
    """x: [B, H, W, 12] -> y: [B, H, W, 4]."""
    B, H, W, _ = x.shape
    y = np.empty((B, H, W, TSURR_COUT), np.float32) if out is None else out
    px, onx, keep = _t._ptr(x, np.float32)
    py, ony, _ = _t._ptr(y, np.float32)
    if onx != ony:
        raise ValueError("x and out must both be host or both be device arrays")
    _t._check(load().tsurr_forward(net, px, int(B), py, onx))
    return y


def tsurr_backward(net, x, target, mask) -> float:
    """Loss of the batch; the gradients stay in the library (tsurr_get_grads)."""
    B = x.shape[0]
    px, on0, k0 = _t._ptr(x, np.float32)
    pt, on1, k1 = _t._ptr(target, np.float32)
    pm, on2, k2 = _t._ptr(mask, np.float32)
    if not on0 == on1 == on2:
        raise ValueError("x, target and mask must all be host or all be device arrays")
    loss = C.c_double(0.0)
    _t._check(load().tsurr_backward(net, px, pt, pm, int(B), C.byref(loss), on0))
    return loss.value


def tsurr_adam(net, lr, beta1=0.9, beta2=0.999, eps=1e-8, t=1):
    _t._check(load().tsurr_adam(net, float(lr), float(beta1), float(beta2), float(eps), int(t)))


def tsurr_sync(net):
    _t._check(load().tsurr_sync(net))


def tsurr_destroy(net):
    if net:
        load().tsurr_destroy(net)


def _dev(t):
    """A contiguous float32 CUDA tensor (the helpers take device arrays only)."""
    if not (hasattr(t, "is_cuda") and t.is_cuda and t.is_contiguous() and str(t.dtype) == "torch.float32"):
        raise TypeError("expected a contiguous float32 CUDA tensor")
    return C.c_void_p(t.data_ptr())


def tsurr_features(height, scalars, out=None, stream=None):
    """Network input x[B,H,W,12] from height maps [B,H,W] and scalars [B,9] (device tensors)."""
    import torch
    B, H, W = height.shape
    if out is None:
        out = torch.empty((B, H, W, 12), dtype=torch.float32, device=height.device)
    _t._check(load().tsurr_features(_dev(height), _dev(scalars), B, H, W, _dev(out), _t._stream_handle(stream)))
    return out


def tsurr_indicator(y, press, out=None, stream=None):
    """Predicted per-frame error sqrt(mean(y[...,3]^2)) / press (device tensors)."""
    import torch
    B, H, W, _ = y.shape
    if out is None:
        out = torch.empty((B,), dtype=torch.float32, device=y.device)
    _t._check(load().tsurr_indicator(_dev(y), _dev(press), B, H, W, _dev(out), _t._stream_handle(stream)))
    return out
