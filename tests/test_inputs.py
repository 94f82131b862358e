"""The seeded input generators (paper_2405_02914_gb300/inputs.py), shared by
the oracle and the CUDA path: the particle lattice, its tags, the
trajectories and the uneven batch have the structure the workloads state."""
import math

import numpy as np
import pytest

from paper_2405_02914_gb300 import inputs as I


def test_gel_particles_stratified_lattice_and_tags():
    gel = I.Gel(6, 5, 3, 0.5e-3, seed=11)
    x, tag = I.gel_particles(gel)
    n = 6 * 5 * 3 * 8
    assert x.shape == (n, 3) and x.dtype == np.float32 and tag.dtype == np.uint32
    # ids are in order in the low bits
    assert np.array_equal(tag & np.uint32(0x0FFFFFFF), np.arange(n, dtype=np.uint32))
    # every cell holds exactly one particle in each of its eight sub-cells
    sub = np.floor(x.astype(np.float64) / (0.5 * gel.dx)).astype(np.int64)
    assert sub.min() == 0 and np.all(sub.max(0) == [11, 9, 5])
    key = (sub[:, 2] * 10 + sub[:, 1]) * 12 + sub[:, 0]
    assert np.unique(key).size == n
    # the bottom tag marks the bottom cell layer; the top tag the upper half of the top layer
    bottom = (tag & I.TAG_BOTTOM) != 0
    top = (tag & I.TAG_TOP) != 0
    z = x[:, 2].astype(np.float64)
    assert np.array_equal(bottom, z < gel.dx)
    assert np.array_equal(top, z >= 2.5 * gel.dx)
    assert top.sum() == 6 * 5 * 4
    # the jitter is seeded: same seed, same lattice; another seed, another
    x2, _ = I.gel_particles(I.Gel(6, 5, 3, 0.5e-3, seed=11))
    x3, _ = I.gel_particles(I.Gel(6, 5, 3, 0.5e-3, seed=12))
    assert np.array_equal(x, x2) and not np.array_equal(x, x3)


def test_rest_state_is_identity():
    v, C, F = I.rest_state(7)
    assert not v.any() and not C.any()
    assert np.array_equal(F.reshape(7, 3, 3), np.broadcast_to(np.eye(3, dtype=np.float32), (7, 3, 3)))


def test_press_slip_rotate_keyframes():
    kf = I.press_slip_rotate((1e-3, 2e-3, 5e-3), 0.4e-3, 0.6e-3, 0.5, 10, 20, 30, slip_dir=(0.0, 1.0))
    assert kf.shape == (4, 5)
    assert list(kf[:, 0]) == [0, 10, 30, 60]
    f32 = lambda a: float(np.float32(a))  # noqa: E731
    assert kf[1, 3] == f32(5e-3 - 0.4e-3)                  # pressed
    assert kf[2, 2] == f32(2e-3 + 0.6e-3) and kf[2, 1] == f32(1e-3)   # slid along y
    assert kf[3, 4] == f32(0.5) and kf[2, 4] == 0.0        # then turned
    with pytest.raises(AssertionError):
        I.keyframes([(0, 0, 0, 0, 0), (0, 0, 0, 0, 0)])    # substeps must increase


def test_uneven_batch_ranges():
    """64 instances: cubes of 4:4:1 cells from 48x48x12 to 128x128x32 (cx a
    multiple of 4) at dx = 0.3125 mm, material and indenter parameters in
    their stated ranges, one time step for the batch (CFL 0.4 of the
    stiffest instance), trajectories that press, slip and turn."""
    sc = I.batch_scenes(64, seed=0)
    assert len(sc) == 64
    dts = {s.solver.dt for s in sc}
    assert len(dts) == 1
    npart = []
    for s in sc:
        g = s.gel
        assert g.dx == 0.3125e-3 and g.cx == g.cy == 4 * g.cz and 12 <= g.cz <= 32
        assert 0.8e5 <= s.mat.E <= 3e5 and 0.40 <= s.mat.nu <= 0.48 and 0.2 <= s.ind.mu <= 1.0
        assert s.ind.kind in (I.SPHERE, I.CYLINDER, I.PRISM, I.PERLIN)
        kf = s.keyframes
        press = kf[0, 3] - kf[1, 3] - 0.37 * g.dx
        assert 0.3e-3 - 1e-9 <= press <= 1.5e-3 + 1e-9
        assert 0.0 <= kf[-1, 4] <= math.radians(45.0) + 1e-6
        assert s.n_substeps == int(kf[-1, 0])
        npart.append(g.n_particles)
        # the stiffest instance sets the step: CFL 0.4 of its P-wave speed
        lam = s.mat.E * s.mat.nu / ((1 + s.mat.nu) * (1 - 2 * s.mat.nu))
        G = s.mat.E / (2 * (1 + s.mat.nu))
        assert s.solver.dt <= 0.4 * g.dx / math.sqrt((lam + 2 * G) / 1100.0) * (1 + 1e-12)
    assert min(npart) >= 48 * 48 * 12 * 8 and max(npart) <= 128 * 128 * 32 * 8
    assert 1.2e6 < np.mean(npart) < 2.1e6                  # mean of the uniform size draw is about 1.6 M
    # seeded: the same seed gives the same batch
    sc2 = I.batch_scenes(64, seed=0)
    assert all(a.gel.cx == b.gel.cx and a.mat.E == b.mat.E for a, b in zip(sc, sc2))


def test_surrogate_batch_shapes_and_mask():
    x, t, m = I.surrogate_batch(3, 2, 16, 24)
    assert x.shape == (2, 16, 24, I.SURR_CIN) and t.shape == (2, 16, 24, 3) and m.shape == (2, 16, 24)
    assert x.dtype == t.dtype == m.dtype == np.float32
    assert set(np.unique(m)) <= {0.0, 1.0} and 0.5 < m.mean() < 0.95
    p = I.surrogate_params(4)
    assert p.size == sum(co * 9 * ci + co for ci, co in I.SURR_CONVS)


def test_object_particles_fill_the_shapes():
    """Lattice points of spacing s inside each shape: the count approaches
    the volume / s^3, every point is inside, and the set is symmetric about
    the indenter frame's centre."""
    import math
    s = 0.1e-3
    sph = I.object_particles(I.sphere(1e-3, 0.5), s)
    assert abs(len(sph) * s ** 3 / (4 / 3 * math.pi * 1e-9) - 1) < 0.03
    assert np.all(np.linalg.norm(sph, axis=1) <= 1e-3 + 1e-12)
    assert np.allclose(np.sort(sph[:, 0]), np.sort(-sph[:, 0]), atol=1e-9)
    bx = I.object_particles(I.box(1e-3, 0.5e-3, 0.5e-3, 0.0, 0.5), s)
    assert len(bx) == 20 * 10 * 10
    cy = I.object_particles(I.cylinder(1e-3, 2e-3, 0.0, 0.5), s)
    assert abs(len(cy) * s ** 3 / (math.pi * 1e-6 * 2e-3) - 1) < 0.03
    sc = I.with_object_particles(I.scene_small())
    dx = sc.gel.dx
    assert sc.ind.obj_m == pytest.approx(sc.mat.rho * dx ** 3 / 8, rel=1e-12)      # an elastomer particle's mass


def test_sensor_leds_face_inward_and_texture_is_contiguous():
    W, H, p, Z = 16, 12, 0.5e-3, 4e-3
    leds = I.sensor_leds(W, H, p, Z)
    centre = np.array([W * p / 2, H * p / 2, Z / 2])
    for c, u, v, rgb in leds:
        e = np.cross(u, v)
        assert (centre - np.array(c)) @ e > 0                  # emits toward the gel
        assert 0 < c[2] - abs(v[2]) and c[2] + abs(v[2]) < Z   # inside the gel's height
    t = I.base_texture(W, H, seed=3)
    assert t.shape == (H, W, 3) and t.dtype == np.float32 and t.flags["C_CONTIGUOUS"]
    assert t.min() >= 0.55 and t.max() <= 0.85
