"""Seeded synthetic scene inputs for the IMPM elastomer substep.

This module holds no arithmetic of the method itself.  It only draws the
inputs that the CUDA path and the FP64 oracle both consume: the jittered
particle lattice of the gel block, particle tags, the node box that bounds
the simulation domain, material constants, indenter geometry, the indenter
pose keyframes and the permutation table of the Perlin-bump indenter.

Geometry conventions (shared by both consumers as *inputs*):

* The gel block occupies [0, cx*dx] x [0, cy*dx] x [0, cz*dx] (metres); its
  base plane is z = 0.  The paper initialises the elastomer as a cuboid of
  particles with the object centred above it (Sec. IV-B).
* The background grid is a box of nodes; node (a, b, c) of the box sits at
  ((a-ox)*dx, (b-oy)*dx, (c-oz)*dx).  The grid fills the simulation space and
  does not move (Sec. III-A).
* Particle id = ((k*cy + j)*cx + i)*8 + s with s = sx + 2*sy + 4*sz the
  stratified 2x2x2 sub-cell of cell (i, j, k).  Tag = id | flag bits.
* An indenter pose is given by its tip (the lowest point of the object,
  the calibration point x_o of Algorithm 1) and a yaw angle about the
  vertical axis through the tip.  The SDF frame centre sits ``tip_offset``
  above the tip.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

TAG_BOTTOM = np.uint32(0x80000000)   # particle starts in the bottom cell layer
TAG_TOP = np.uint32(0x40000000)      # particle starts in the upper half of the top cell layer
TAG_MARKER = np.uint32(0x20000000)   # embedded marker particle
ID_MASK = np.uint32(0x1FFFFFFF)

SPHERE, CYLINDER, BOX, PRISM, PERLIN, NONE = 0, 1, 2, 3, 4, -1
BASE_FIXED, BASE_SLIP, BASE_FREE = 0, 1, 2

NODE_PAD = 4          # nodes below 0 in x, y, z
TOP_HEADROOM = 8      # nodes above the gel top before the +z wall


def _round_up(a: int, m: int) -> int:
    return (a + m - 1) // m * m


@dataclasses.dataclass
class Gel:
    """Gel block, its particle lattice and the node box around it."""
    cx: int
    cy: int
    cz: int
    dx: float
    seed: int = 0
    ppc: int = 8

    @property
    def n_particles(self) -> int:
        return self.cx * self.cy * self.cz * self.ppc

    @property
    def origin(self):
        return (NODE_PAD, NODE_PAD, NODE_PAD)

    @property
    def nodes(self):
        """Node box dims (nx, ny, nz), rounded up to whole 4-node blocks."""
        return (_round_up(self.cx + 2 * NODE_PAD, 4), _round_up(self.cy + 2 * NODE_PAD, 4),
                _round_up(self.cz + NODE_PAD + TOP_HEADROOM, 4))

    @property
    def height(self) -> float:
        return self.cz * self.dx


@dataclasses.dataclass
class Material:
    E: float = 1.5e5
    nu: float = 0.45
    rho: float = 1100.0
    gravity: tuple = (0.0, 0.0, -9.81)


@dataclasses.dataclass
class Indenter:
    """Rigid indenter: shape code, 8 shape parameters, friction, tip offset,
    and optionally a kinetic friction coefficient mu_k <= mu for the slip
    (0: the slip uses mu too).

    params by shape (metres):
      SPHERE   [r]
      CYLINDER [r, h, edge_round]              axis vertical, flat face down
      BOX      [hx, hy, hz, edge_round]        half sizes
      PRISM    [side, length, edge_round]      equilateral section, apex down,
                                               extruded along the local x axis
      PERLIN   [hx, hy, hz, edge_round, amp, period, persistence, octaves]
    """
    kind: int
    params: Sequence[float]
    mu: float
    tip_offset: float
    perm: np.ndarray = dataclasses.field(default_factory=lambda: np.arange(256, dtype=np.int32))
    mu_k: float = 0.0
    obj: Optional[np.ndarray] = None      # object particles (indenter frame), or None: SDF contact
    obj_m: float = 0.0                    # mass of one object particle

    def params8(self) -> np.ndarray:
        p = np.zeros(8, dtype=np.float64)
        p[:len(self.params)] = self.params
        return p


def sphere(r: float, mu: float) -> Indenter:
    return Indenter(SPHERE, [r], mu, r)


def cylinder(r: float, h: float, rnd: float, mu: float) -> Indenter:
    return Indenter(CYLINDER, [r, h, rnd], mu, h / 2)


def box(hx: float, hy: float, hz: float, rnd: float, mu: float) -> Indenter:
    return Indenter(BOX, [hx, hy, hz, rnd], mu, hz)


def prism(side: float, length: float, rnd: float, mu: float) -> Indenter:
    inr = side / (2.0 * math.sqrt(3.0))          # inradius of the section
    return Indenter(PRISM, [side, length, rnd], mu, 2.0 * inr - rnd)


def perlin_plate(hx: float, hy: float, hz: float, rnd: float, amp: float,
                 period: float, persistence: float, octaves: int, mu: float,
                 seed: int) -> Indenter:
    perm = np.random.Generator(np.random.Philox(key=seed + 0x5EED)).permutation(256).astype(np.int32)
    return Indenter(PERLIN, [hx, hy, hz, rnd, amp, period, persistence, float(octaves)],
                    mu, hz, perm)


def object_particles(ind: Indenter, spacing: float) -> np.ndarray:
    """Points of a lattice of the given spacing (cell centres, symmetric about
    the indenter frame's centre) inside the solid indenter, in the indenter
    frame: sphere, cylinder (flat faces horizontal) and box, with their edge
    rounding.  The object of the particle-represented indenter."""
    p = ind.params
    if ind.kind == SPHERE:
        ext = np.array([p[0]] * 3)
    elif ind.kind == CYLINDER:
        ext = np.array([p[0], p[0], p[1] / 2])
    elif ind.kind == BOX:
        ext = np.array(p[:3], dtype=np.float64)
    else:
        raise ValueError("object particles for sphere, cylinder and box indenters")
    axes = [(np.arange(-int(np.ceil(e / spacing)), int(np.ceil(e / spacing))) + 0.5) * spacing for e in ext]
    q = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, 3)
    if ind.kind == SPHERE:
        inside = np.linalg.norm(q, axis=1) <= p[0]
    elif ind.kind == CYLINDER:
        r, rnd = p[0], p[2]
        d = np.stack([np.hypot(q[:, 0], q[:, 1]) - (r - rnd), np.abs(q[:, 2]) - (p[1] / 2 - rnd)], 1)
        inside = np.linalg.norm(np.maximum(d, 0.0), axis=1) <= rnd
    else:
        rnd = p[3]
        d = np.abs(q) - (ext - rnd)
        inside = np.linalg.norm(np.maximum(d, 0.0), axis=1) <= rnd
    return q[inside].astype(np.float32)


def with_object_particles(scene: "Scene", per_cell: int = 8) -> "Scene":
    """The scene with its indenter represented by particles (the paper's own
    coupling): per_cell (8) particles per grid cell at the gel's density, so
    each carries the mass of an elastomer particle."""
    spacing = scene.gel.dx / round(per_cell ** (1.0 / 3.0))
    ind = dataclasses.replace(scene.ind)
    ind.obj = object_particles(ind, spacing)
    ind.obj_m = float(scene.mat.rho * spacing ** 3)
    return dataclasses.replace(scene, ind=ind, name=scene.name + "+objparticles")


def sensor_leds(W: int, H: int, pitch: float, gel_height: float, colors: str = "gelsight"):
    """Four LED panels on the side faces of the gel under a W x H readout of
    the given pitch, each spanning its face and 5-95 % of the gel's height
    (inside the gel: no panel edge at the membrane's height, where a path's
    first step would meet it edge-on) and emitting inward (the emitting
    side of u x v): (centre, u, v, rgb) tuples.  colors: "gelsight" (red, green, blue, white radiance 1) or
    "white" (all four white, as in the slip and rotation sensor)."""
    X, Y, Z = W * pitch, H * pitch, gel_height
    rgb = ([(1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0), (1.0, 1.0, 1.0)] if colors == "gelsight"
           else [(1.0, 1.0, 1.0)] * 4)
    hz = (0.0, 0.0, 0.45 * Z)
    return [((0.0, Y / 2, Z / 2), (0.0, Y / 2, 0.0), hz, rgb[0]),          # x = 0, emits +x
            ((X, Y / 2, Z / 2), (0.0, -Y / 2, 0.0), hz, rgb[1]),           # x = X, emits -x
            ((X / 2, 0.0, Z / 2), (-X / 2, 0.0, 0.0), hz, rgb[2]),         # y = 0, emits +y
            ((X / 2, Y, Z / 2), (X / 2, 0.0, 0.0), hz, rgb[3])]            # y = Y, emits -y


def base_texture(W: int, H: int, seed: int = 0) -> np.ndarray:
    """Synthetic (H, W, 3) albedo in [0.55, 0.85] (the real sensors' base
    images are not available): smooth seeded blotches."""
    rng = np.random.Generator(np.random.Philox(key=seed + 0x7E47))
    a = rng.uniform(0.0, 1.0, (H // 8 + 2, W // 8 + 2, 3))
    yy = np.clip((np.arange(H) + 0.5) / 8.0, 0, a.shape[0] - 1.001)
    xx = np.clip((np.arange(W) + 0.5) / 8.0, 0, a.shape[1] - 1.001)
    i0, j0 = yy.astype(int), xx.astype(int)
    fy, fx = (yy - i0)[:, None, None], (xx - j0)[None, :, None]
    t = ((1 - fy) * ((1 - fx) * a[i0][:, j0] + fx * a[i0][:, j0 + 1]) +
         fy * ((1 - fx) * a[i0 + 1][:, j0] + fx * a[i0 + 1][:, j0 + 1]))
    return np.ascontiguousarray(0.55 + 0.3 * t, dtype=np.float32)


def no_indenter() -> Indenter:
    return Indenter(NONE, [], 0.0, 0.0)


@dataclasses.dataclass
class Solver:
    dt: float
    relrest_limit: int = 8           # 1 reduces IMPM to plain MPM
    relrest_threshold: float = 0.5
    base_mode: int = BASE_FIXED
    walls: int = 1


@dataclasses.dataclass
class Scene:
    gel: Gel
    mat: Material
    ind: Indenter
    keyframes: np.ndarray            # (n, 5) float64: substep, tip x, y, z, yaw
    solver: Solver
    readout_every: int = 100
    readout_px: int = 128
    readout_pitch: float = 0.0
    n_substeps: int = 0
    name: str = ""
    meta: dict = dataclasses.field(default_factory=dict)


# ---------------------------------------------------------------- particles

def gel_particles(gel: Gel):
    """Jittered 2x2x2-stratified lattice (8 per cell), float32 SoA-ready.

    Returns (x [n,3] float32, tag [n] uint32) in particle-id order.  The
    jitter draws one uniform in [0,1) per particle and axis from a Philox
    stream keyed by the gel seed, in id order.
    """
    assert gel.ppc == 8
    cx, cy, cz, dx = gel.cx, gel.cy, gel.cz, gel.dx
    n = gel.n_particles
    x = np.empty((n, 3), dtype=np.float32)
    tag = np.empty(n, dtype=np.uint32)
    rng = np.random.Generator(np.random.Philox(key=gel.seed))
    per_layer = cx * cy * 8
    s = np.arange(8)
    sx, sy, sz = s & 1, (s >> 1) & 1, (s >> 2) & 1
    jj, ii = np.meshgrid(np.arange(cy), np.arange(cx), indexing="ij")
    ii = ii.reshape(-1)
    jj = jj.reshape(-1)
    for k in range(cz):
        u = rng.random((per_layer, 3))
        ci = np.repeat(ii, 8)
        cj = np.repeat(jj, 8)
        ssx = np.tile(sx, cx * cy)
        ssy = np.tile(sy, cx * cy)
        ssz = np.tile(sz, cx * cy)
        lo = k * per_layer
        x[lo:lo + per_layer, 0] = ((ci + (ssx + u[:, 0]) * 0.5) * dx).astype(np.float32)
        x[lo:lo + per_layer, 1] = ((cj + (ssy + u[:, 1]) * 0.5) * dx).astype(np.float32)
        x[lo:lo + per_layer, 2] = ((k + (ssz + u[:, 2]) * 0.5) * dx).astype(np.float32)
        ids = np.arange(lo, lo + per_layer, dtype=np.uint32)
        t = ids.copy()
        if k == 0:
            t |= TAG_BOTTOM
        if k == cz - 1:
            t[ssz == 1] |= TAG_TOP
        tag[lo:lo + per_layer] = t
    return x, tag


def marker_ids(gel: Gel, m: int = 16) -> np.ndarray:
    """Ids of an m x m array of top-layer particles (sub-cell sx=sy=0, sz=1)."""
    out = np.empty(m * m, dtype=np.int64)
    for a in range(m):
        for b in range(m):
            i = min(gel.cx - 1, int((b + 0.5) * gel.cx / m))
            j = min(gel.cy - 1, int((a + 0.5) * gel.cy / m))
            k = gel.cz - 1
            out[a * m + b] = ((k * gel.cy + j) * gel.cx + i) * 8 + 4
    return out


def tag_markers(tag: np.ndarray, ids: np.ndarray) -> np.ndarray:
    t = tag.copy()
    t[ids] |= TAG_MARKER
    return t


def rest_state(n: int):
    """Zero velocity, zero affine field, identity deformation gradient."""
    v = np.zeros((n, 3), dtype=np.float32)
    C = np.zeros((n, 9), dtype=np.float32)
    F = np.zeros((n, 9), dtype=np.float32)
    F[:, 0] = F[:, 4] = F[:, 8] = 1.0
    return v, C, F


# ---------------------------------------------------------------- trajectories

def keyframes(rows: List[Sequence[float]]) -> np.ndarray:
    kf = np.asarray(rows, dtype=np.float64).reshape(-1, 5)
    # the CUDA side consumes float32 poses; round here so both read the same values
    kf[:, 1:] = kf[:, 1:].astype(np.float32).astype(np.float64)
    assert np.all(np.diff(kf[:, 0]) > 0), "keyframe substeps must increase"
    return kf


def press_slip_rotate(tip0, press, slip, rotate, n_press, n_slip, n_rot, slip_dir=(1.0, 0.0)):
    x0, y0, z0 = tip0
    z1 = z0 - press
    x2, y2 = x0 + slip * slip_dir[0], y0 + slip * slip_dir[1]
    rows = [(0, x0, y0, z0, 0.0), (n_press, x0, y0, z1, 0.0)]
    s = n_press
    if n_slip > 0:
        s += n_slip
        rows.append((s, x2, y2, z1, 0.0))
    if n_rot > 0:
        s += n_rot
        rows.append((s, x2, y2, z1, rotate))
    return keyframes(rows)


# ---------------------------------------------------------------- named workloads

def scene_press65k(dt: float = 2e-5) -> Scene:
    """Plain press: 20x20x5 mm block, 32x32x8 cells, 65,536 particles, r=4 mm
    sphere pressing 0.5 mm over 500 substeps, mu=0.6, readout every 50."""
    gel = Gel(32, 32, 8, 0.625e-3, seed=1)
    H = gel.height
    n = int(round(500 * 2e-5 / dt))
    kf = press_slip_rotate((10e-3, 10e-3, H), 0.5e-3, 0.0, 0.0, n, 0, 0)
    return Scene(gel, Material(), sphere(4e-3, 0.6), kf, Solver(dt=dt),
                 readout_every=n // 10, readout_px=32, readout_pitch=gel.dx,
                 n_substeps=n, name="press65k")


def scene_pad4m(seed: int = 0, dt: float = 5e-6) -> Scene:
    """Sensor pad press-slip-rotate: 128x128x32 cells at dx=0.3125 mm
    (40x40x10 mm, 4,194,304 particles), indenter drawn by seed from
    {sphere r5, cylinder r3 h10, cube 6}, 0.25 mm edge rounding, press 1 mm
    over 5,000 substeps, slip 3 mm over 7,500, rotate 30 deg over 7,500,
    mu=0.5, 128x128 readout every 100 substeps."""
    gel = Gel(128, 128, 32, 0.3125e-3, seed=seed + 2)
    H = gel.height
    pick = seed % 3
    if pick == 0:
        ind = sphere(5e-3, 0.5)
    elif pick == 1:
        ind = cylinder(3e-3, 10e-3, 0.25e-3, 0.5)
    else:
        ind = box(3e-3, 3e-3, 3e-3, 0.25e-3, 0.5)
    kf = press_slip_rotate((20e-3, 20e-3, H), 1.0e-3, 3e-3, math.radians(30.0),
                           5000, 7500, 7500)
    return Scene(gel, Material(), ind, kf, Solver(dt=dt), readout_every=100,
                 readout_px=128, readout_pitch=gel.dx, n_substeps=20000, name="pad4m")


def scene_large33m(dt: float = 4e-6, gap: float = 0.0) -> Scene:
    """Large gel: 60x60x15 mm on 256x256x64 cells (33,554,432 particles),
    Perlin-bump plate, press 1 mm / slip 3 mm / rotate 90 deg over 50,000
    substeps, 16x16 markers every 200 substeps.  ``gap`` (in cells) starts
    the tip that far above the gel top, at the same press speed (parity
    scenes use 0.37 so that the plate's flat face is not on a node plane)."""
    gel = Gel(256, 256, 64, 0.234375e-3, seed=5)
    H = gel.height
    ind = perlin_plate(4e-3, 4e-3, 1e-3, 0.25e-3, 0.3e-3, 4e-3, 0.5, 4, 0.5, seed=5)
    g = gap * gel.dx
    n_gap = int(round(10000 * g / 1.0e-3))
    kf = press_slip_rotate((30e-3, 30e-3, H + g), 1.0e-3 + g, 3e-3, math.radians(90.0),
                           10000 + n_gap, 20000, 20000)
    return Scene(gel, Material(), ind, kf, Solver(dt=dt), readout_every=200,
                 readout_px=128, readout_pitch=60e-3 / 128, n_substeps=50000,
                 name="large33m")


def scene_small(cx=16, cy=16, cz=4, dx=0.625e-3, kind=SPHERE, mu=0.6, press=0.15e-3,
                slip=0.0, rotate=0.0, n_press=100, n_slip=0, n_rot=0, dt=1e-5,
                limit=8, seed=7, E=1.5e5, nu=0.45, gap=0.37) -> Scene:
    """A small scene of the same structure, for parity tests (indenter speeds
    of the order of 0.1 m/s, like the press workloads).  The tip starts
    ``gap`` cells above the gel so that a flat indenter face never sits on a
    node plane at a substep (where an FP32 and an FP64 contact test of the
    same node may legitimately disagree)."""
    gel = Gel(cx, cy, cz, dx, seed=seed)
    H = gel.height
    r = 0.3 * min(cx, cy) * dx
    if kind == SPHERE:
        ind = sphere(r, mu)
    elif kind == CYLINDER:
        ind = cylinder(r * 0.6, 2 * r, 2.5 * dx, mu)
    elif kind == BOX:
        # edge rounding beyond the deepest contact node: interior normals of a
        # box jump on its medial surface, where FP32 and FP64 may pick
        # different faces for the same node
        ind = box(r * 0.6, r * 0.6, r * 0.6, 2.5 * dx, mu)
    elif kind == PRISM:
        ind = prism(1.2 * r, 1.6 * r, 0.4 * dx, mu)
    elif kind == PERLIN:
        ind = perlin_plate(r * 0.7, r * 0.7, 0.3 * r, 0.4 * dx, 0.1 * r, 0.8 * r, 0.5, 4, mu, seed)
    else:
        ind = no_indenter()
    kf = press_slip_rotate((cx * dx / 2, cy * dx / 2, H + gap * dx), press + gap * dx, slip, rotate,
                           n_press, n_slip, n_rot)
    return Scene(gel, Material(E=E, nu=nu), ind, kf, Solver(dt=dt, relrest_limit=limit),
                 readout_every=max(1, (n_press + n_slip + n_rot) // 4),
                 readout_px=cx, readout_pitch=dx,
                 n_substeps=n_press + n_slip + n_rot, name="small")


def batch_scenes(n: int = 64, seed: int = 0, scale: float = 1.0) -> List[Scene]:
    """Uneven batch: grids 48x48x12 .. 128x128x32 (4:4:1, cx a multiple of 4),
    dx = 0.3125 mm, E in [0.8,3]e5 Pa, nu in [0.40,0.48], mu in [0.2,1.0],
    indenters from {sphere, cylinder, prism, Perlin plate}, press 0.3-1.5 mm,
    slip 0-4 mm, rotation 0-45 deg.  ``scale`` < 1 shrinks the grids for
    quick tests."""
    rng = np.random.Generator(np.random.Philox(key=0xBA7C + seed))
    dx = 0.3125e-3
    out = []
    for b in range(n):
        lo, hi = 12, 32
        cz = int(rng.integers(lo, hi + 1))
        cz = max(2, int(round(cz * scale)))
        cx = 4 * cz
        E = float(rng.uniform(0.8e5, 3e5))
        nu = float(rng.uniform(0.40, 0.48))
        mu = float(rng.uniform(0.2, 1.0))
        kind = int(rng.integers(0, 4))
        press = float(rng.uniform(0.3e-3, 1.5e-3)) * scale
        slip = float(rng.uniform(0.0, 4e-3)) * scale
        rot = math.radians(float(rng.uniform(0.0, 45.0)))
        gel = Gel(cx, cx, cz, dx, seed=1000 + seed * 131 + b)
        H = gel.height
        L = cx * dx
        if kind == 0:
            ind = sphere(min(5e-3, 0.25 * L), mu)
        elif kind == 1:
            ind = cylinder(min(3e-3, 0.15 * L), 10e-3, 0.25e-3, mu)
        elif kind == 2:
            ind = prism(min(6e-3, 0.3 * L), min(10e-3, 0.5 * L), 0.25e-3, mu)
        else:
            ind = perlin_plate(min(4e-3, 0.2 * L), min(4e-3, 0.2 * L), 1e-3, 0.25e-3,
                               0.3e-3 * scale, 4e-3 * scale, 0.5, 4, mu, seed=seed * 977 + b)
        lam = E * nu / ((1 + nu) * (1 - 2 * nu))
        G = E / (2 * (1 + nu))
        c = math.sqrt((lam + 2 * G) / 1100.0)
        out.append((gel, Material(E=E, nu=nu), ind, press, slip, rot, c))
    c_max = max(o[6] for o in out)
    dt = 0.4 * dx / c_max
    scenes = []
    for gel, mat, ind, press, slip, rot, _ in out:
        n_press = max(1, int(math.ceil(press / (0.2 * dt))))
        n_slip = int(math.ceil(slip / (0.2 * dt))) if slip > 0 else 0
        n_rot = int(math.ceil(rot / (40.0 * dt))) if rot > 0 else 0
        L = gel.cx * gel.dx
        # the tip starts 0.37 dx above the gel so that no flat face sits on a node plane
        gap = 0.37 * gel.dx
        kf = press_slip_rotate((L / 2 - slip / 2, L / 2, gel.height + gap), press + gap, slip, rot,
                               n_press, n_slip, n_rot)
        scenes.append(Scene(gel, mat, ind, kf, Solver(dt=dt), readout_every=100,
                            readout_px=gel.cx, readout_pitch=gel.dx,
                            n_substeps=n_press + n_slip + n_rot, name="batch"))
    return scenes


# ------------------------------------------------------------------ surface surrogate inputs

# (cin, cout) of the surrogate's nine 3x3 convolutions in parameter order; the
# first layer's 16 inputs hold 12 real channels, the last layer's 16 rows 4 real ones
SURR_CONVS = [(16, 32), (32, 64), (64, 128), (128, 256), (256, 256), (256, 128), (128, 64), (64, 32), (32, 16)]
SURR_CIN, SURR_COUT = 12, 4


def surrogate_params(seed: int, bias_std: float = 0.0, scale_last: float = 0.1) -> np.ndarray:
    """Flat FP32 parameter vector, layer by layer W[cout][3][3][cin] then b[cout]:
    He-normal weights on the real channels (the last layer scaled by
    ``scale_last``), zero on the padded ones, biases N(0, bias_std)."""
    rng = np.random.Generator(np.random.Philox(key=0x5A77 + seed))
    parts = []
    last = len(SURR_CONVS) - 1
    for li, (cin, cout) in enumerate(SURR_CONVS):
        rin = SURR_CIN if li == 0 else cin
        rout = SURR_COUT if li == last else cout
        w = np.zeros((cout, 3, 3, cin), np.float32)
        std = math.sqrt(2.0 / (9 * rin)) * (scale_last if li == last else 1.0)
        w[:rout, :, :, :rin] = rng.standard_normal((rout, 3, 3, rin)) * std
        b = np.zeros(cout, np.float32)
        if bias_std > 0:
            b[:rout] = rng.standard_normal(rout) * bias_std
        parts += [w.ravel(), b]
    return np.concatenate(parts).astype(np.float32)


def surrogate_batch(seed: int, B: int, H: int, W: int, mask_frac: float = 0.8):
    """Random features x[B,H,W,12] (one smooth bump channel, eleven per-sample
    constants), targets t[B,H,W,3] and a 0/1 mask[B,H,W] covering a centred
    window of about ``mask_frac`` of each side."""
    rng = np.random.Generator(np.random.Philox(key=0x5B47 + seed))
    x = np.empty((B, H, W, SURR_CIN), np.float32)
    yy, xx = np.meshgrid(np.linspace(-1, 1, H), np.linspace(-1, 1, W), indexing="ij")
    for b in range(B):
        cy, cx, r = rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5), rng.uniform(0.2, 0.6)
        x[b, :, :, 0] = np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / (r * r))
        x[b, :, :, 1:] = rng.standard_normal(SURR_CIN - 1).astype(np.float32)
    t = (rng.standard_normal((B, H, W, 3)) * 0.5).astype(np.float32)
    m = np.zeros((B, H, W), np.float32)
    my, mx = int(round(H * (1 - mask_frac) / 2)), int(round(W * (1 - mask_frac) / 2))
    m[:, my:H - my, mx:W - mx] = 1.0
    return x, t, m


# surrogate dataset pads: 64 x 64 x 16 cells at dx = 0.3125 mm (20 x 20 x 5 mm,
# 524,288 particles); a 128 x 128 pixel window at pitch dx/2 is the whole pad
SURR_PAD = (64, 64, 16)
SURR_DX = 0.3125e-3
SURR_PX = 128
SURR_PHASES = (800, 2400, 2000)      # substeps of the press, slip and rotate phases


def surrogate_scenes(n: int, seed: int, first: int = 0) -> List[Scene]:
    """Trajectories ``first .. first+n-1`` of the seeded surrogate dataset
    (seed picks the split: training and held-out sets use different seeds).
    Each draws E in [0.8,3]e5 Pa, nu in [0.40,0.47], mu in [0.2,1.0], an
    indenter from {sphere r 3-5 mm, cylinder r 2-3 mm, prism side 4-6 mm,
    Perlin plate 8 x 8 mm, amplitude 0.3 mm} (edges rounded to 2 dx),
    press 0.3-1.0 mm, slip 0-3 mm in
    a random direction and rotation of -45..45 deg, over fixed phase lengths
    so that every trajectory of a batch has the same substep count.  All pads
    share one particle lattice (gel seed 0) so one reference configuration
    serves all."""
    cx, cy, cz = SURR_PAD
    dx = SURR_DX
    gel = Gel(cx, cy, cz, dx, seed=0)
    L = cx * dx
    # common step from the stiffest material of the ranges (CFL 0.3); flat
    # punches into gels with nu = 0.48 at CFL 0.4 inverted cells within the
    # press phase, so nu stops at 0.47 here
    E, nu = 3e5, 0.47
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    G = E / (2 * (1 + nu))
    dt = 0.3 * dx / math.sqrt((lam + 2 * G) / 1100.0)
    n_press, n_slip, n_rot = SURR_PHASES
    out = []
    for k in range(first, first + n):
        rng = np.random.Generator(np.random.Philox(key=0x5C3A + 7919 * seed + k))
        Em = float(rng.uniform(0.8e5, 3e5))
        num = float(rng.uniform(0.40, 0.47))
        mu = float(rng.uniform(0.2, 1.0))
        kind = int(rng.integers(0, 4))
        press = float(rng.uniform(0.3e-3, 1.0e-3))
        slip = float(rng.uniform(0.0, 3e-3))
        ang = float(rng.uniform(0.0, 2 * math.pi))
        rot = math.radians(float(rng.uniform(-45.0, 45.0)))
        # edges rounded to 2 dx: a sharper rim under a nearly incompressible gel
        # (nu -> 0.48) with sticking friction inverted cells in early runs
        rnd = 2.0 * dx
        if kind == 0:
            ind = sphere(float(rng.uniform(3e-3, 5e-3)), mu)
        elif kind == 1:
            ind = cylinder(float(rng.uniform(2e-3, 3e-3)), 10e-3, rnd, mu)
        elif kind == 2:
            ind = prism(float(rng.uniform(4e-3, 6e-3)), float(rng.uniform(6e-3, 10e-3)), rnd, mu)
        else:
            ind = perlin_plate(4e-3, 4e-3, 1e-3, rnd, 0.3e-3, 4e-3, 0.5, 4, mu, seed=7919 * seed + k)
        gap = 0.37 * dx
        d = (math.cos(ang), math.sin(ang))
        tip0 = (L / 2 - 0.5 * slip * d[0], L / 2 - 0.5 * slip * d[1], gel.height + gap)
        kf = press_slip_rotate(tip0, press + gap, slip, rot, n_press, n_slip, n_rot, slip_dir=d)
        meta = dict(press=press, gap=gap, slip=slip, slip_dir=d, rotate=rot, E=Em, nu=num, mu=mu, kind=kind)
        out.append(Scene(gel, Material(E=Em, nu=num), ind, kf, Solver(dt=dt), readout_every=100,
                         readout_px=SURR_PX, readout_pitch=dx / 2, n_substeps=n_press + n_slip + n_rot,
                         name="surrogate", meta=meta))
    return out
