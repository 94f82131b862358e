"""ctypes binding of the FP64 C oracle (impm_oracle.c).

Test infrastructure only: tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg use it; the product path never imports it.  Every function
here marshals numpy arrays; the arithmetic lives in impm_oracle.c.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "impm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
               "-o", tmp, _SRC, "-lm"]
        try:    # OpenMP for orc_run_par (all host cores); without it the same code runs on one
            subprocess.check_call(cmd[:-1] + ["-fopenmp", "-lm"], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Scene(C.Structure):
    _fields_ = [("cx", C.c_int), ("cy", C.c_int), ("cz", C.c_int),
                ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("ox", C.c_int), ("oy", C.c_int), ("oz", C.c_int),
                ("base_mode", C.c_int), ("walls", C.c_int), ("limit", C.c_int), ("ppc", C.c_int),
                ("pad_", C.c_int),
                ("dx", C.c_double), ("dt", C.c_double), ("rho", C.c_double),
                ("E", C.c_double), ("nu", C.c_double), ("g", C.c_double * 3),
                ("threshold", C.c_double)]


class Indenter(C.Structure):
    _fields_ = [("kind", C.c_int), ("pad_", C.c_int), ("p", C.c_double * 8),
                ("mu", C.c_double), ("tip_offset", C.c_double), ("perm", C.c_int * 256),
                ("mu_k", C.c_double), ("obj_q", C.POINTER(C.c_double)), ("n_obj", C.c_long),
                ("obj_m", C.c_double)]


class Pose(C.Structure):
    _fields_ = [("tip", C.c_double * 3), ("c", C.c_double * 3), ("yaw", C.c_double),
                ("cs", C.c_double), ("sn", C.c_double), ("vlin", C.c_double * 3),
                ("omega", C.c_double)]


_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_U = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_I = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.POINTER
            L.orc_weights.argtypes = [C.c_double, C.c_double, P(C.c_int), _D]
            L.orc_kirchhoff.argtypes = [_D, C.c_double, C.c_double, _D]
            L.orc_kirchhoff.restype = C.c_int
            L.orc_pose_eval.argtypes = [_D, C.c_int, C.c_int, C.c_double, C.c_double, P(Pose)]
            L.orc_sdf_local.argtypes = [P(Indenter), _D, _D]
            L.orc_sdf_local.restype = C.c_double
            L.orc_sdf.argtypes = [P(Indenter), P(Pose), _D, _D]
            L.orc_sdf.restype = C.c_double
            L.orc_p2g.argtypes = [P(Scene), C.c_int, _D, _D, _D, _D, _D, _D]
            L.orc_p2g.restype = C.c_int
            L.orc_grid_update.argtypes = [P(Scene), P(Indenter), P(Pose), _D, _D, _D, P(C.c_long)]
            L.orc_object_p2g.argtypes = [P(Scene), P(Indenter), P(Pose), _D, _D]
            L.orc_object_p2g.restype = C.c_int
            L.orc_grid_update.restype = C.c_int
            L.orc_g2p.argtypes = [P(Scene), C.c_int, _D, _U, _D, _D, _D]
            L.orc_g2p.restype = C.c_int
            L.orc_nearest.argtypes = [C.c_int, _D, _D]
            L.orc_nearest.restype = C.c_int
            L.orc_relrest_accept.argtypes = [P(Scene), P(Indenter), P(Pose), _D, _D]
            L.orc_relrest_accept.restype = C.c_int
            L.orc_substep.argtypes = [P(Scene), P(Indenter), _D, C.c_int, C.c_int, C.c_int,
                                      _D, _D, _D, _D, _U, _D, _D, _D, P(C.c_int), P(C.c_int),
                                      P(C.c_long)]
            L.orc_substep.restype = C.c_int
            L.orc_run.argtypes = [P(Scene), P(Indenter), _D, C.c_int, C.c_int, C.c_int, C.c_int,
                                  _D, _D, _D, _D, _U, _I, _I]
            L.orc_run.restype = C.c_int
            L.orc_run_par.argtypes = [P(Scene), P(Indenter), _D, C.c_int, C.c_int, C.c_int, C.c_int,
                                      _D, _D, _D, _D, _U, _I, _I, C.c_int]
            L.orc_run_par.restype = C.c_int
            L.orc_threads.restype = C.c_int
            L.orc_surface.argtypes = [C.c_int, _D, _U, C.c_int, C.c_int, C.c_double, C.c_double,
                                      _D, _D]
            L.orc_surface_disp.argtypes = [C.c_int, _D, _D, _U, C.c_int, C.c_int, C.c_double, _D]
            L.orc_indenter_height.argtypes = [P(Indenter), P(Pose), C.c_double, C.c_int, C.c_int, C.c_double,
                                              C.c_double, C.c_double, _D]
            _lib = L
    return _lib


ERRORS = {0: "ok", 1: "particle left the node box", 2: "non-finite state or J <= 0", 3: "bad argument"}


class OracleError(RuntimeError):
    pass


def _check(rc):
    if rc != 0:
        raise OracleError(ERRORS.get(rc, str(rc)))


# ----------------------------------------------------------------- descriptors

def make_scene(scene) -> Scene:
    """Scene struct from an inputs.Scene."""
    g = scene.gel
    nx, ny, nz = g.nodes
    ox, oy, oz = g.origin
    s = Scene()
    s.cx, s.cy, s.cz = g.cx, g.cy, g.cz
    s.nx, s.ny, s.nz = nx, ny, nz
    s.ox, s.oy, s.oz = ox, oy, oz
    s.base_mode = scene.solver.base_mode
    s.walls = scene.solver.walls
    s.limit = scene.solver.relrest_limit
    s.ppc = g.ppc
    s.dx = g.dx
    s.dt = scene.solver.dt
    s.rho = scene.mat.rho
    s.E = scene.mat.E
    s.nu = scene.mat.nu
    for a in range(3):
        s.g[a] = scene.mat.gravity[a]
    s.threshold = scene.solver.relrest_threshold
    return s


def make_indenter(ind) -> Indenter:
    o = Indenter()
    o.kind = ind.kind
    p = ind.params8()
    for a in range(8):
        o.p[a] = p[a]
    o.mu = ind.mu
    o.tip_offset = ind.tip_offset
    perm = np.asarray(ind.perm, dtype=np.int32)
    for a in range(256):
        o.perm[a] = int(perm[a])
    o.mu_k = ind.mu_k
    if getattr(ind, "obj", None) is not None and len(ind.obj):
        q = np.ascontiguousarray(ind.obj, dtype=np.float64).reshape(-1)
        o._obj_keep = q                       # the C struct points into this array
        o.obj_q = q.ctypes.data_as(C.POINTER(C.c_double))
        o.n_obj = q.size // 3
        o.obj_m = ind.obj_m
    return o


# ----------------------------------------------------------------- functions

def weights(xp: float, dx: float):
    b = C.c_int(0)
    w = np.zeros(3)
    lib().orc_weights(float(xp), float(dx), C.byref(b), w)
    return b.value, w


def kirchhoff(F, mu: float, lam: float):
    tau = np.zeros(9)
    _check(lib().orc_kirchhoff(np.ascontiguousarray(F, dtype=np.float64).reshape(9), mu, lam, tau))
    return tau.reshape(3, 3)


def pose(kf, k: int, dt: float, tip_offset: float) -> Pose:
    p = Pose()
    kf = np.ascontiguousarray(kf, dtype=np.float64)
    lib().orc_pose_eval(kf, kf.shape[0], int(k), float(dt), float(tip_offset), C.byref(p))
    return p


def sdf_local(ind: Indenter, q):
    g = np.zeros(3)
    phi = lib().orc_sdf_local(C.byref(ind), np.ascontiguousarray(q, dtype=np.float64), g)
    return phi, g


def sdf(ind: Indenter, ps: Pose, xw):
    n = np.zeros(3)
    phi = lib().orc_sdf(C.byref(ind), C.byref(ps), np.ascontiguousarray(xw, dtype=np.float64), n)
    return phi, n


class State:
    """FP64 particle state in id order."""

    def __init__(self, x, v, C_, F, tag):
        self.x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
        self.v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1, 3)
        self.C = np.ascontiguousarray(C_, dtype=np.float64).reshape(-1, 9)
        self.F = np.ascontiguousarray(F, dtype=np.float64).reshape(-1, 9)
        self.tag = np.ascontiguousarray(tag, dtype=np.uint32)

    @property
    def n(self):
        return self.x.shape[0]

    def copy(self):
        return State(self.x.copy(), self.v.copy(), self.C.copy(), self.F.copy(), self.tag.copy())


def n_nodes(s: Scene) -> int:
    return s.nx * s.ny * s.nz


def p2g(s: Scene, st: State):
    nn = n_nodes(s)
    M = np.zeros(nn)
    MG = np.zeros(3 * nn)
    _check(lib().orc_p2g(C.byref(s), st.n, st.x, st.v, st.C, st.F, M, MG))
    return M, MG.reshape(-1, 3)


def object_p2g(s: Scene, ind: Indenter, ps: Pose, M=None, MG=None):
    """The object particles' P2G added to (copies of) M, MG (zeros if None)."""
    nn = n_nodes(s)
    M = np.zeros(nn) if M is None else np.array(M, dtype=np.float64)
    MG = np.zeros(3 * nn) if MG is None else np.array(MG, dtype=np.float64).reshape(-1)
    _check(lib().orc_object_p2g(C.byref(s), C.byref(ind), C.byref(ps), M, MG))
    return M, MG.reshape(-1, 3)


def grid_update(s: Scene, ind: Indenter, ps: Pose, M, MG):
    nn = n_nodes(s)
    V = np.zeros(3 * nn)
    cnt = C.c_long(0)
    _check(lib().orc_grid_update(C.byref(s), C.byref(ind), C.byref(ps),
                                 np.ascontiguousarray(M, dtype=np.float64),
                                 np.ascontiguousarray(MG, dtype=np.float64).reshape(-1), V,
                                 C.byref(cnt)))
    return V.reshape(-1, 3), cnt.value


def g2p(s: Scene, st: State, V):
    v = np.zeros((st.n, 3))
    Cm = np.zeros((st.n, 9))
    _check(lib().orc_g2p(C.byref(s), st.n, st.x, st.tag,
                         np.ascontiguousarray(V, dtype=np.float64).reshape(-1), v, Cm))
    return v, Cm


def nearest(x, xo) -> int:
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    return lib().orc_nearest(x.shape[0], x, np.ascontiguousarray(xo, dtype=np.float64))


def relrest_accept(s: Scene, ind: Indenter, ps: Pose, xe, ve) -> bool:
    """Algorithm 1's relative-rest check at the calibration particle x_e with
    velocity v_e (True: accept the pass)."""
    return bool(lib().orc_relrest_accept(C.byref(s), C.byref(ind), C.byref(ps),
                                         np.ascontiguousarray(xe, dtype=np.float64),
                                         np.ascontiguousarray(ve, dtype=np.float64)))


def substep(s: Scene, ind: Indenter, kf, k: int, st: State):
    """One IMPM time step in place; returns (passes, x_e index, contact nodes)."""
    nn = n_nodes(s)
    M = np.zeros(nn)
    MG = np.zeros(3 * nn)
    V = np.zeros(3 * nn)
    ps, e, nc = C.c_int(0), C.c_int(0), C.c_long(0)
    kf = np.ascontiguousarray(kf, dtype=np.float64)
    _check(lib().orc_substep(C.byref(s), C.byref(ind), kf, kf.shape[0], int(k), st.n,
                             st.x, st.v, st.C, st.F, st.tag, M, MG, V,
                             C.byref(ps), C.byref(e), C.byref(nc)))
    return ps.value, e.value, nc.value


def run(s: Scene, ind: Indenter, kf, k0: int, nsub: int, st: State):
    """Substeps k0..k0+nsub-1 in place; returns (passes per substep, x_e per substep)."""
    kf = np.ascontiguousarray(kf, dtype=np.float64)
    pl = np.zeros(max(nsub, 1), dtype=np.int32)
    el = np.zeros(max(nsub, 1), dtype=np.int32)
    _check(lib().orc_run(C.byref(s), C.byref(ind), kf, kf.shape[0], int(k0), int(nsub), st.n,
                         st.x, st.v, st.C, st.F, st.tag, pl, el))
    return pl[:nsub], el[:nsub]


def threads() -> int:
    """Threads run_par uses by default (the host's cores with OpenMP, else 1)."""
    return int(lib().orc_threads())


def run_par(s: Scene, ind: Indenter, kf, k0: int, nsub: int, st: State, nthreads: int = 0):
    """run() with its loops shared among nthreads host threads (0: all);
    the grid sums are added per thread chunk, so results equal run()'s to
    rounding.  Returns (passes per substep, x_e per substep)."""
    kf = np.ascontiguousarray(kf, dtype=np.float64)
    pl = np.zeros(max(nsub, 1), dtype=np.int32)
    el = np.zeros(max(nsub, 1), dtype=np.int32)
    _check(lib().orc_run_par(C.byref(s), C.byref(ind), kf, kf.shape[0], int(k0), int(nsub), st.n,
                             st.x, st.v, st.C, st.F, st.tag, pl, el, int(nthreads)))
    return pl[:nsub], el[:nsub]


def surface(st: State, W: int, H: int, pitch: float, h_empty: float):
    h = np.zeros(W * H)
    nrm = np.zeros(W * H * 3)
    lib().orc_surface(st.n, st.x, st.tag, W, H, float(pitch), float(h_empty), h, nrm)
    return h.reshape(H, W), nrm.reshape(H, W, 3)


def lame(E: float, nu: float):
    return E / (2 * (1 + nu)), E * nu / ((1 + nu) * (1 - 2 * nu))


def surface_disp(st: State, xref, W: int, H: int, pitch: float):
    """Displacement of the top layer splatted at the reference positions."""
    u = np.zeros(W * H * 3)
    xref = np.ascontiguousarray(xref, dtype=np.float64).reshape(-1, 3)
    lib().orc_surface_disp(st.n, st.x, xref, st.tag, W, H, float(pitch), u)
    return u.reshape(H, W, 3)


def indenter_height(ind: Indenter, ps: Pose, gel_height: float, W: int, H: int, pitch: float, clip: float,
                    step: float):
    h = np.zeros(W * H)
    lib().orc_indenter_height(C.byref(ind), C.byref(ps), float(gel_height), W, H, float(pitch), float(clip),
                              float(step), h)
    return h.reshape(H, W)
