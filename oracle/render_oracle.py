"""ctypes binding of the FP64 C oracle of the sensor image (render_oracle.c).

TEST INFRASTRUCTURE ONLY: used by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py, never by the product path.  Nothing here
computes: arrays are marshalled to render_oracle.c.
"""
import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "render_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc_render.so")
_lock = threading.Lock()
_lib = None
MAX_LIGHTS = 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Desc(C.Structure):
    _fields_ = [("c", (C.c_double * 3) * MAX_LIGHTS), ("u", (C.c_double * 3) * MAX_LIGHTS),
                ("v", (C.c_double * 3) * MAX_LIGHTS), ("L", (C.c_double * 3) * MAX_LIGHTS),
                ("n_lights", C.c_int), ("spp", C.c_int), ("max_bounces", C.c_int), ("pad_", C.c_int),
                ("z_floor", C.c_double), ("seed", C.c_uint64)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            _D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
            L.ro_uniform.argtypes = [C.c_uint64, C.c_uint64]
            L.ro_uniform.restype = C.c_double
            L.ro_render.argtypes = [_D, _D, C.c_int, C.c_int, C.c_double, C.POINTER(Desc), _D]
            L.ro_render.restype = C.c_int
            L.ro_mse_psnr.argtypes = [_D, _D, C.c_long, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.ro_mse_psnr.restype = None
            L.ro_ssim.argtypes = [_D, _D, C.c_int, C.c_int, C.c_int, C.c_double, C.POINTER(C.c_double)]
            L.ro_ssim.restype = C.c_int
            _lib = L
    return _lib


def make_desc(leds, spp, max_bounces, z_floor, seed) -> Desc:
    """leds: up to four (centre, u, v, rgb) tuples (metres, radiance)."""
    d = Desc()
    d.n_lights = len(leds)
    for k, (c, u, v, L) in enumerate(leds):
        for a in range(3):
            d.c[k][a], d.u[k][a], d.v[k][a], d.L[k][a] = c[a], u[a], v[a], L[a]
    d.spp, d.max_bounces, d.z_floor, d.seed = int(spp), int(max_bounces), float(z_floor), int(seed)
    return d


def uniform(seed: int, counter: int) -> float:
    return lib().ro_uniform(seed, counter)


def render(height, albedo, pitch, desc: Desc):
    """(H, W, 3) image of the height field (H, W) with the albedo (H, W, 3)."""
    h = np.ascontiguousarray(height, dtype=np.float64)
    H, W = h.shape
    a = np.ascontiguousarray(np.broadcast_to(albedo, (H, W, 3)), dtype=np.float64)
    out = np.zeros((H, W, 3))
    if lib().ro_render(h, a.reshape(-1), W, H, pitch, C.byref(desc), out.reshape(-1)) != 0:
        raise ValueError("bad render arguments")
    return out


def mse_psnr(a, b, max_value):
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    b = np.ascontiguousarray(b, dtype=np.float64).reshape(-1)
    m, p = C.c_double(), C.c_double()
    lib().ro_mse_psnr(a, b, a.size, max_value, C.byref(m), C.byref(p))
    return m.value, p.value


def ssim(a, b, max_value):
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    if a.ndim == 2:
        a, b = a[..., None], b[..., None]
    H, W, Cc = a.shape
    s = C.c_double()
    if lib().ro_ssim(a.reshape(-1), b.reshape(-1), W, H, Cc, max_value, C.byref(s)) != 0:
        raise ValueError("images must be at least 11 x 11")
    return s.value
