"""Python binding of libtsim.so (include/tsim.h): argument marshalling only.

Every step of the simulation runs in the library's CUDA kernels.  This
module converts numpy arrays (host, ``on_device=0``) or torch CUDA tensors
(device, ``on_device=1``) into pointers, fills the descriptor structs, and
raises ``TsimError`` on a non-zero status.  There is no CPU fallback: if the
library cannot be built or loaded, ``load()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

TSIM_OK = 0
ERRORS = {1: "TSIM_ERR_INVALID_ARG", 2: "TSIM_ERR_OOM", 3: "TSIM_ERR_CUDA", 4: "TSIM_ERR_NUMERIC",
          5: "TSIM_ERR_DOMAIN", 6: "TSIM_ERR_CAPACITY", 7: "TSIM_ERR_STATE",
          8: "TSIM_ERR_TIMEOUT"}

EXPORTS = ["tsim_create", "tsim_set_solver", "tsim_set_indenter", "tsim_set_trajectory",
           "tsim_write_particles", "tsim_set_substep", "tsim_step", "tsim_read_particles",
           "tsim_read_grid", "tsim_read_surface", "tsim_read_markers", "tsim_read_log", "tsim_sync",
           "tsim_stats", "tsim_use_graph", "tsim_profile", "tsim_kernel_time", "tsim_pass_time", "tsim_last_error",
           "tsim_block_slots", "tsim_destroy", "tsim_p2g_noalloc", "tsim_read_displacement", "tsim_read_indenter_height",
           "tsim_set_tuning", "tsim_get_tuning", "tsim_autotune", "tsim_set_object_particles", "tsim_render",
           "tsim_image_metrics"]


class TsimError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (ERRORS.get(code, code), msg))
        self.code = code


class GelDesc(C.Structure):
    _fields_ = [("cx", C.c_int), ("cy", C.c_int), ("cz", C.c_int), ("nx", C.c_int), ("ny", C.c_int),
                ("nz", C.c_int), ("ox", C.c_int), ("oy", C.c_int), ("oz", C.c_int), ("ppc", C.c_int),
                ("dx", C.c_float)]


class MaterialDesc(C.Structure):
    _fields_ = [("E", C.c_float), ("nu", C.c_float), ("rho", C.c_float), ("gravity", C.c_float * 3)]


class IndenterDesc(C.Structure):
    _fields_ = [("kind", C.c_int), ("p", C.c_float * 8), ("mu", C.c_float), ("tip_offset", C.c_float),
                ("perm", C.c_int32 * 256), ("mu_kinetic", C.c_float)]


class Keyframe(C.Structure):
    _fields_ = [("substep", C.c_int32), ("tip", C.c_float * 3), ("yaw", C.c_float)]


class SolverDesc(C.Structure):
    _fields_ = [("dt", C.c_float), ("relrest_limit", C.c_int), ("relrest_threshold", C.c_float),
                ("base_mode", C.c_int), ("walls", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("substeps", C.c_int64), ("passes", C.c_int64), ("particle_updates", C.c_int64),
                ("status", C.c_uint32), ("n_inst", C.c_int32), ("spilled", C.c_int64), ("spill_max", C.c_int32),
                ("pad_", C.c_int32)]


MAX_LEDS = 4


class RenderDesc(C.Structure):
    _fields_ = [("c", (C.c_float * 3) * MAX_LEDS), ("u", (C.c_float * 3) * MAX_LEDS),
                ("v", (C.c_float * 3) * MAX_LEDS), ("L", (C.c_float * 3) * MAX_LEDS),
                ("n_lights", C.c_int), ("spp", C.c_int), ("max_bounces", C.c_int), ("z_floor", C.c_float),
                ("seed", C.c_uint64)]


def render_desc(leds, spp=128, max_bounces=4, z_floor=0.0, seed=0) -> RenderDesc:
    """leds: up to four (centre, u, v, rgb) tuples (see inputs.sensor_leds)."""
    d = RenderDesc()
    d.n_lights = len(leds)
    for k, (c, u, v, L) in enumerate(leds):
        for a in range(3):
            d.c[k][a], d.u[k][a], d.v[k][a], d.L[k][a] = c[a], u[a], v[a], L[a]
    d.spp, d.max_bounces, d.z_floor, d.seed = int(spp), int(max_bounces), float(z_floor), int(seed)
    return d


class Tuning(C.Structure):
    _fields_ = [("grid_threads", C.c_int), ("grid_flat", C.c_int), ("graph_chunk", C.c_int),
                ("us_per_mupdate", C.c_float)]

    def as_dict(self):
        return {"grid_threads": self.grid_threads, "grid_flat": self.grid_flat, "graph_chunk": self.graph_chunk,
                "us_per_mupdate": self.us_per_mupdate}


_lib = None


def load():
    """Build (if stale) and load libtsim.so; raises if that is impossible."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P, vp = C.POINTER, C.c_void_p
        sig = {
            "tsim_create": (C.c_int, [C.c_int, P(GelDesc), P(MaterialDesc), vp, P(vp)]),
            "tsim_set_solver": (C.c_int, [vp, P(SolverDesc)]),
            "tsim_set_indenter": (C.c_int, [vp, C.c_int, P(IndenterDesc)]),
            "tsim_set_trajectory": (C.c_int, [vp, C.c_int, vp, C.c_int, C.c_int]),
            "tsim_write_particles": (C.c_int, [vp, C.c_int, vp, vp, vp, vp, vp, C.c_int, C.c_int]),
            "tsim_set_substep": (C.c_int, [vp, C.c_int64]),
            "tsim_step": (C.c_int, [vp, C.c_int]),
            "tsim_read_particles": (C.c_int, [vp, C.c_int, vp, vp, vp, vp, C.c_int, C.c_int]),
            "tsim_read_grid": (C.c_int, [vp, C.c_int, vp, C.c_int]),
            "tsim_read_surface": (C.c_int, [vp, C.c_int, vp, vp, C.c_int, C.c_int, C.c_float, C.c_int]),
            "tsim_read_markers": (C.c_int, [vp, C.c_int, vp, C.c_int, vp, C.c_int]),
            "tsim_read_displacement": (C.c_int, [vp, C.c_int, vp, vp, C.c_int, C.c_int, C.c_float, C.c_int]),
            "tsim_read_indenter_height": (C.c_int, [vp, C.c_int, vp, C.c_int, C.c_int, C.c_float, C.c_float,
                                                    C.c_int]),
            "tsim_read_log": (C.c_int, [vp, C.c_int, vp, vp, C.c_int]),
            "tsim_sync": (C.c_int, [vp]),
            "tsim_stats": (C.c_int, [vp, P(Stats)]),
            "tsim_use_graph": (C.c_int, [vp, C.c_int]),
            "tsim_profile": (C.c_int, [vp, C.c_int]),
            "tsim_kernel_time": (C.c_int, [vp, P(C.c_int64), P(C.c_double)]),
            "tsim_pass_time": (C.c_int, [vp, P(C.c_int64), P(C.c_double), P(C.c_double)]),
            "tsim_last_error": (C.c_char_p, []),
            "tsim_block_slots": (C.c_int, []),
            "tsim_destroy": (None, [vp]),
            "tsim_p2g_noalloc": (C.c_int, [P(GelDesc), P(MaterialDesc), C.c_float, vp, vp, vp, vp, C.c_int,
                                           vp, vp]),
            "tsim_set_tuning": (C.c_int, [vp, P(Tuning)]),
            "tsim_set_object_particles": (C.c_int, [vp, C.c_int, vp, C.c_int, C.c_float, C.c_int]),
            "tsim_render": (C.c_int, [vp, vp, C.c_int, C.c_int, C.c_float, P(RenderDesc), vp, vp]),
            "tsim_image_metrics": (C.c_int, [vp, vp, C.c_int, C.c_int, C.c_int, C.c_float, P(C.c_double), vp]),
            "tsim_get_tuning": (C.c_int, [vp, P(Tuning)]),
            "tsim_autotune": (C.c_int, [vp, C.c_int, P(Tuning)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def lib_path() -> str:
    return _build.LIB


def _check(rc):
    if rc != TSIM_OK:
        raise TsimError(rc, load().tsim_last_error().decode())


def _ptr(a, dtype):
    """(pointer, on_device, keepalive) for a numpy array or a torch CUDA tensor."""
    if a is None:
        return None, 0, None
    if hasattr(a, "data_ptr"):                      # torch tensor
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        on = 1 if a.is_cuda else 0
        return C.c_void_p(a.data_ptr()), on, a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data_as(C.c_void_p), 0, arr


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


# ------------------------------------------------------------------ descriptors from inputs

def gel_desc(gel) -> GelDesc:
    g = GelDesc()
    g.cx, g.cy, g.cz = gel.cx, gel.cy, gel.cz
    g.nx, g.ny, g.nz = gel.nodes
    g.ox, g.oy, g.oz = gel.origin
    g.ppc = gel.ppc
    g.dx = gel.dx
    return g


def material_desc(mat) -> MaterialDesc:
    m = MaterialDesc()
    m.E, m.nu, m.rho = mat.E, mat.nu, mat.rho
    for a in range(3):
        m.gravity[a] = mat.gravity[a]
    return m


def indenter_desc(ind) -> IndenterDesc:
    o = IndenterDesc()
    o.kind = ind.kind
    p = ind.params8()
    for a in range(8):
        o.p[a] = p[a]
    o.mu = ind.mu
    o.tip_offset = ind.tip_offset
    perm = np.asarray(ind.perm, dtype=np.int32)
    for a in range(256):
        o.perm[a] = int(perm[a])
    o.mu_kinetic = ind.mu_k
    return o


def keyframes(kf) -> "C.Array":
    kf = np.asarray(kf, dtype=np.float64).reshape(-1, 5)
    arr = (Keyframe * kf.shape[0])()
    for a, row in enumerate(kf):
        arr[a].substep = int(row[0])
        for d in range(3):
            arr[a].tip[d] = row[1 + d]
        arr[a].yaw = row[4]
    return arr


def solver_desc(s) -> SolverDesc:
    o = SolverDesc()
    o.dt = s.dt
    o.relrest_limit = s.relrest_limit
    o.relrest_threshold = s.relrest_threshold
    o.base_mode = s.base_mode
    o.walls = s.walls
    return o


# ------------------------------------------------------------------ same-name calls

def tsim_create(gels, mats, stream=None):
    L = load()
    n = len(gels)
    G = (GelDesc * n)(*gels)
    M = (MaterialDesc * n)(*mats)
    out = C.c_void_p()
    _check(L.tsim_create(n, G, M, _stream_handle(stream), C.byref(out)))
    return out


def tsim_set_solver(ctx, solver: SolverDesc):
    _check(load().tsim_set_solver(ctx, C.byref(solver)))


def tsim_set_indenter(ctx, inst, ind: IndenterDesc):
    _check(load().tsim_set_indenter(ctx, inst, C.byref(ind)))


def tsim_render(height, albedo, pitch, desc: RenderDesc, out=None, stream=None):
    """(H, W, 3) sensor image of the (H, W) height field (CUDA tensors)."""
    import torch
    H, W = height.shape
    for t in (height, albedo) + ((out,) if out is not None else ()):
        if not t.is_contiguous() or t.dtype != torch.float32:
            raise ValueError("height, albedo and out must be contiguous float32 tensors")
    if tuple(albedo.shape) != (H, W, 3):
        raise ValueError("albedo must be (H, W, 3)")
    if out is None:
        out = torch.empty((H, W, 3), dtype=torch.float32, device=height.device)
    _check(load().tsim_render(C.c_void_p(height.data_ptr()), C.c_void_p(albedo.data_ptr()), int(W), int(H),
                              float(pitch), C.byref(desc), C.c_void_p(out.data_ptr()), _stream_handle(stream)))
    return out


def tsim_image_metrics(a, b, max_value=1.0, stream=None):
    """(MSE, PSNR, SSIM) of two (H, W, C) or (H, W) CUDA tensors."""
    import torch
    H, W = a.shape[:2]
    Cc = a.shape[2] if a.dim() == 3 else 1
    if not (a.is_contiguous() and b.is_contiguous()) or a.shape != b.shape or a.dtype != torch.float32 or \
            b.dtype != torch.float32:
        raise ValueError("a and b must be contiguous float32 tensors of one shape")
    out = (C.c_double * 3)()
    _check(load().tsim_image_metrics(C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr()), int(W), int(H), int(Cc),
                                     float(max_value), out, _stream_handle(stream)))
    return out[0], out[1], out[2]


def tsim_set_object_particles(ctx, inst, q, mass):
    """q: (n, 3) object particles in the indenter frame (numpy or CUDA
    tensor, float32), each of the given mass; n = 0 (or None) returns to the
    SDF contact."""
    if q is None or len(q) == 0:
        _check(load().tsim_set_object_particles(ctx, inst, None, 0, 0.0, 0))
        return
    p, on, keep = _ptr(q, np.float32)
    _check(load().tsim_set_object_particles(ctx, inst, p, int(len(q)), float(mass), on))


def tsim_set_trajectory(ctx, inst, kf):
    arr = kf if isinstance(kf, C.Array) else keyframes(kf)
    _check(load().tsim_set_trajectory(ctx, inst, C.cast(arr, C.c_void_p), len(arr), 0))


def tsim_write_particles(ctx, inst, x, v, Cm, F, tag):
    px, on, kx = _ptr(x, np.float32)
    pv, _, kv = _ptr(v, np.float32)
    pc, _, kc = _ptr(Cm, np.float32)
    pf, _, kF = _ptr(F, np.float32)
    pt, _, kt = _ptr(tag, np.uint32)
    n = int(np.prod(x.shape) // 3)
    _check(load().tsim_write_particles(ctx, inst, px, pv, pc, pf, pt, n, on))


def tsim_set_substep(ctx, k):
    _check(load().tsim_set_substep(ctx, int(k)))


def tsim_step(ctx, n):
    _check(load().tsim_step(ctx, int(n)))


def tsim_read_particles(ctx, inst, n, out=None):
    """Returns (x, v, C, F) as numpy arrays, or fills the given torch tensors."""
    if out is None:
        x = np.empty((n, 3), np.float32); v = np.empty((n, 3), np.float32)
        Cm = np.empty((n, 9), np.float32); F = np.empty((n, 9), np.float32)
        arrs = (x, v, Cm, F)
    else:
        arrs = out
    ptrs = [_ptr(a, np.float32) for a in arrs]
    on = ptrs[0][1]
    _check(load().tsim_read_particles(ctx, inst, ptrs[0][0], ptrs[1][0], ptrs[2][0], ptrs[3][0], n, on))
    return arrs


def tsim_read_grid(ctx, inst, n_nodes, out=None):
    arr = np.empty((n_nodes, 4), np.float32) if out is None else out
    p, on, _ = _ptr(arr, np.float32)
    _check(load().tsim_read_grid(ctx, inst, p, on))
    return arr


def tsim_read_surface(ctx, inst, W, H, pitch, height=None, normal=None):
    h = np.empty((H, W), np.float32) if height is None else height
    n = np.empty((H, W, 3), np.float32) if normal is None else normal
    ph, on, _ = _ptr(h, np.float32)
    pn, _, _ = _ptr(n, np.float32)
    _check(load().tsim_read_surface(ctx, inst, ph, pn, int(W), int(H), float(pitch), on))
    return h, n


def tsim_read_displacement(ctx, inst, x_ref, W, H, pitch, out=None):
    arr = np.empty((H, W, 3), np.float32) if out is None else out
    pr, onr, keep = _ptr(x_ref, np.float32)
    p, on, _ = _ptr(arr, np.float32)
    if onr != on:
        raise ValueError("x_ref and out must both be host or both be device arrays")
    _check(load().tsim_read_displacement(ctx, inst, pr, p, int(W), int(H), float(pitch), on))
    return arr


def tsim_read_indenter_height(ctx, inst, W, H, pitch, clip, out=None):
    arr = np.empty((H, W), np.float32) if out is None else out
    p, on, _ = _ptr(arr, np.float32)
    _check(load().tsim_read_indenter_height(ctx, inst, p, int(W), int(H), float(pitch), float(clip), on))
    return arr


def tsim_read_markers(ctx, inst, ids, out=None):
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    arr = np.empty((ids.shape[0], 3), np.float32) if out is None else out
    p, on, _ = _ptr(arr, np.float32)
    _check(load().tsim_read_markers(ctx, inst, ids.ctypes.data_as(C.c_void_p), ids.shape[0], p, on))
    return arr


def tsim_read_log(ctx, inst, n):
    passes = np.zeros(n, np.int32)
    calib = np.zeros(n, np.int32)
    _check(load().tsim_read_log(ctx, inst, passes.ctypes.data_as(C.c_void_p),
                                calib.ctypes.data_as(C.c_void_p), n))
    return passes, calib


def tsim_sync(ctx):
    _check(load().tsim_sync(ctx))


def tsim_stats(ctx) -> Stats:
    s = Stats()
    _check(load().tsim_stats(ctx, C.byref(s)))
    return s


def tsim_use_graph(ctx, enable):
    _check(load().tsim_use_graph(ctx, 1 if enable else 0))


def tsim_profile(ctx, enable):
    _check(load().tsim_profile(ctx, 1 if enable else 0))


def tsim_kernel_time(ctx):
    n = C.c_int64()
    ms = C.c_double()
    _check(load().tsim_kernel_time(ctx, C.byref(n), C.byref(ms)))
    return n.value, ms.value


def tsim_pass_time(ctx):
    """(commit launches, commit ms, repeat-pass loop ms) since the last reset."""
    n = C.c_int64()
    ms = C.c_double()
    lms = C.c_double()
    _check(load().tsim_pass_time(ctx, C.byref(n), C.byref(ms), C.byref(lms)))
    return n.value, ms.value, lms.value


def tsim_set_tuning(ctx, grid_threads=256, grid_flat=0, graph_chunk=20):
    t = Tuning(int(grid_threads), int(grid_flat), int(graph_chunk), 0.0)
    _check(load().tsim_set_tuning(ctx, C.byref(t)))


def tsim_get_tuning(ctx) -> dict:
    t = Tuning()
    _check(load().tsim_get_tuning(ctx, C.byref(t)))
    return t.as_dict()


def tsim_autotune(ctx, n) -> dict:
    """Advance n substeps (as tsim_step) while choosing the fastest launch configuration."""
    t = Tuning()
    _check(load().tsim_autotune(ctx, int(n), C.byref(t)))
    return t.as_dict()


def tsim_destroy(ctx):
    if ctx:
        load().tsim_destroy(ctx)


def tsim_block_slots() -> int:
    """Particle slots of one 4x4x4-cell block (the rest spill)."""
    return int(load().tsim_block_slots())


# ------------------------------------------------------------------ convenience wrapper

class Sim:
    """A context built from ``inputs.Scene`` objects (one instance each)."""

    def __init__(self, scenes, stream=None, use_graph=False, states=None):
        from . import inputs
        if not isinstance(scenes, (list, tuple)):
            scenes = [scenes]
        self.scenes = list(scenes)
        self.ctx = tsim_create([gel_desc(s.gel) for s in scenes], [material_desc(s.mat) for s in scenes],
                               stream)
        tsim_set_solver(self.ctx, solver_desc(scenes[0].solver))
        for i, s in enumerate(scenes):
            tsim_set_indenter(self.ctx, i, indenter_desc(s.ind))
            if getattr(s.ind, "obj", None) is not None:
                tsim_set_object_particles(self.ctx, i, s.ind.obj, s.ind.obj_m)
            tsim_set_trajectory(self.ctx, i, s.keyframes)
        for i, s in enumerate(scenes):
            if states is not None and states[i] is not None:
                x, v, Cm, F, tag = states[i]
            else:
                x, tag = inputs.gel_particles(s.gel)
                v, Cm, F = inputs.rest_state(x.shape[0])
            tsim_write_particles(self.ctx, i, x, v, Cm, F, tag)
        if use_graph:
            tsim_use_graph(self.ctx, True)

    def n_particles(self, i=0):
        return self.scenes[i].gel.n_particles

    def n_nodes(self, i=0):
        nx, ny, nz = self.scenes[i].gel.nodes
        return nx * ny * nz

    def step(self, n):
        tsim_step(self.ctx, n)

    def particles(self, i=0):
        return tsim_read_particles(self.ctx, i, self.n_particles(i))

    def grid(self, i=0):
        return tsim_read_grid(self.ctx, i, self.n_nodes(i))

    def surface(self, i=0, W=None, H=None, pitch=None):
        s = self.scenes[i]
        W = W or s.readout_px
        H = H or s.readout_px
        pitch = pitch or s.readout_pitch or s.gel.dx
        return tsim_read_surface(self.ctx, i, W, H, pitch)

    def log(self, n, i=0):
        return tsim_read_log(self.ctx, i, n)

    def stats(self):
        return tsim_stats(self.ctx)

    def close(self):
        if self.ctx:
            tsim_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
