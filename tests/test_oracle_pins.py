"""Pins of the FP64 oracle against what the mathematics fixes.

Each test checks the oracle (oracle/impm_oracle.c) against a closed form, an
invariant or a library routine -- never against a retyped copy of its own
formula -- chosen so that a dropped term, a wrong sign or index, or a
transposed operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2405_02914_gb300 import inputs as I

RNG = np.random.default_rng(1234)


def _scene(cx=8, cy=8, cz=4, dx=1e-3, E=1.5e5, nu=0.45, g=(0.0, 0.0, -9.81), kind=I.NONE,
           mu=0.5, base=I.BASE_FIXED, dt=1e-5, limit=8, seed=3, ind=None):
    gel = I.Gel(cx, cy, cz, dx, seed=seed)
    if ind is None:
        ind = I.no_indenter() if kind == I.NONE else I.sphere(0.3 * cx * dx, mu)
    kf = I.keyframes([(0, cx * dx / 2, cy * dx / 2, 10.0, 0.0)])
    return I.Scene(gel, I.Material(E=E, nu=nu, gravity=g), ind, kf,
                   I.Solver(dt=dt, relrest_limit=limit, base_mode=base))


def _state(scene, v=None, C=None, F=None):
    x, tag = I.gel_particles(scene.gel)
    v0, C0, F0 = I.rest_state(x.shape[0])
    return O.State(x, v0 if v is None else v, C0 if C is None else C, F0 if F is None else F, tag)


def _psi(F, mu, lam):
    """Compressible Neo-Hookean strain energy density."""
    F = F.reshape(3, 3)
    J = np.linalg.det(F)
    return 0.5 * mu * (np.trace(F.T @ F) - 3.0) - mu * np.log(J) + 0.5 * lam * np.log(J) ** 2


# ------------------------------------------------------------------ weights (Eq. 1 kernel)

def test_bspline_moments():
    """Quadratic B-spline: partition of unity, zero first moment, second
    moment dx^2/4 -- the identities behind the 4/W^2 factor of Eqs. 4 and 7."""
    dx = 0.37e-3
    for xp in RNG.uniform(0.0, 40 * dx, 500):
        b, w = O.weights(xp, dx)
        d = (b + np.arange(3)) * dx - xp
        assert abs(w.sum() - 1.0) < 1e-14
        assert abs((w * d).sum()) < 1e-15
        assert abs((w * d * d).sum() - dx * dx / 4.0) < 1e-13 * dx * dx
        assert np.all(w >= 0.0)
        assert 0.5 <= xp / dx - b < 1.5


# ------------------------------------------------------------------ stress (S_p of Eq. 4)

def test_kirchhoff_rest_is_zero():
    mu, lam = O.lame(1.5e5, 0.45)
    assert np.abs(O.kirchhoff(np.eye(3), mu, lam)).max() == 0.0


def test_kirchhoff_is_energy_derivative():
    """tau = (dPsi/dF) F^T, by central differences of the Neo-Hookean energy."""
    mu, lam = O.lame(1.5e5, 0.45)
    for _ in range(10):
        F = np.eye(3) + 0.15 * RNG.standard_normal((3, 3))
        h = 1e-6
        P = np.zeros((3, 3))
        for a in range(3):
            for b in range(3):
                Fp = F.copy(); Fp[a, b] += h
                Fm = F.copy(); Fm[a, b] -= h
                P[a, b] = (_psi(Fp, mu, lam) - _psi(Fm, mu, lam)) / (2 * h)
        tau_fd = P @ F.T
        tau = O.kirchhoff(F, mu, lam)
        assert np.abs(tau - tau_fd).max() < 1e-6 * np.abs(tau_fd).max()


def test_kirchhoff_rotation_covariance():
    mu, lam = O.lame(2e5, 0.4)
    for _ in range(5):
        F = np.eye(3) + 0.2 * RNG.standard_normal((3, 3))
        Q, _ = np.linalg.qr(RNG.standard_normal((3, 3)))
        if np.linalg.det(Q) < 0:
            Q[:, 0] *= -1
        lhs = O.kirchhoff(Q @ F, mu, lam)
        rhs = Q @ O.kirchhoff(F, mu, lam) @ Q.T
        assert np.abs(lhs - rhs).max() < 1e-9 * np.abs(rhs).max()


def test_kirchhoff_small_strain_is_hooke():
    mu, lam = O.lame(1.5e5, 0.45)
    e = 1e-6 * RNG.standard_normal((3, 3))
    e = 0.5 * (e + e.T)
    tau = O.kirchhoff(np.eye(3) + e, mu, lam)
    hooke = lam * np.trace(e) * np.eye(3) + 2 * mu * e
    assert np.abs(tau - hooke).max() < 1e-4 * np.abs(hooke).max()


# ------------------------------------------------------------------ P2G (Eqs. 1-4)

def _random_state(sc):
    st = _state(sc)
    n = st.n
    st.v[:] = 0.05 * RNG.standard_normal((n, 3))
    st.C[:] = 20.0 * RNG.standard_normal((n, 9))
    st.F[:] = (np.eye(3) + 0.05 * RNG.standard_normal((n, 3, 3))).reshape(n, 9)
    return st


def test_p2g_conserves_mass_and_momentum():
    sc = _scene()
    s = O.make_scene(sc)
    st = _random_state(sc)
    M, MG = O.p2g(s, st)
    mp = sc.mat.rho * sc.gel.dx ** 3 / 8
    assert abs(M.sum() - st.n * mp) < 1e-12 * st.n * mp
    # affine and stress terms have zero first moment: total momentum = sum m v
    ref = mp * st.v.sum(axis=0)
    scale = mp * np.abs(st.v).sum()
    assert np.abs(MG.sum(axis=0) - ref).max() < 1e-12 * scale


def test_p2g_apic_angular_momentum():
    """Grid angular momentum = sum_p m x_p x v_p + m dx^2/4 eps_abc C_cb
    (the APIC angular momentum; symmetric stress adds none)."""
    sc = _scene()
    s = O.make_scene(sc)
    st = _random_state(sc)
    M, MG = O.p2g(s, st)
    nx, ny, nz = sc.gel.nodes
    ox, oy, oz = sc.gel.origin
    dx = sc.gel.dx
    az, ay, ax = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    xi = np.stack([(ax - ox) * dx, (ay - oy) * dx, (az - oz) * dx], -1).reshape(-1, 3)
    Lg = np.cross(xi, MG).sum(axis=0)
    mp = sc.mat.rho * dx ** 3 / 8
    Cm = st.C.reshape(-1, 3, 3)
    eps = np.zeros((3, 3, 3))
    eps[0, 1, 2] = eps[1, 2, 0] = eps[2, 0, 1] = 1
    eps[0, 2, 1] = eps[2, 1, 0] = eps[1, 0, 2] = -1
    Lp = mp * np.cross(st.x, st.v).sum(axis=0) + mp * dx * dx / 4 * np.einsum("abc,pcb->a", eps, Cm)
    scale = np.abs(mp * np.cross(st.x, st.v)).sum() + np.abs(mp * dx * dx / 4 * Cm).sum()
    assert np.abs(Lg - Lp).max() < 1e-11 * scale


def test_affine_field_transfers_exactly():
    """v = A x + b, C = A, F = I: P2G gives V_i = A x_i + b on active nodes and
    G2P returns v = A x_p + b and C = A (mass factor and outer-product
    orientation of Eqs. 3 and 7)."""
    sc = _scene(g=(0.0, 0.0, 0.0), base=I.BASE_FREE)
    s = O.make_scene(sc)
    st = _state(sc)
    A = 30.0 * RNG.standard_normal((3, 3))
    b = 0.02 * RNG.standard_normal(3)
    st.v[:] = st.x @ A.T + b
    st.C[:] = np.tile(A.reshape(9), (st.n, 1))
    M, MG = O.p2g(s, st)
    ps = O.pose(sc.keyframes, 0, sc.solver.dt, 0.0)
    V, _ = O.grid_update(s, O.make_indenter(sc.ind), ps, M, MG)
    nx, ny, nz = sc.gel.nodes
    ox, oy, oz = sc.gel.origin
    dx = sc.gel.dx
    az, ay, ax = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    xi = np.stack([(ax - ox) * dx, (ay - oy) * dx, (az - oz) * dx], -1).reshape(-1, 3)
    act = M > 0
    Vref = xi @ A.T + b
    sv = np.abs(Vref[act]).max()
    assert np.abs(V[act] - Vref[act]).max() < 1e-11 * sv
    v, Cm = O.g2p(s, st, V)
    assert np.abs(v - st.v).max() < 1e-11 * sv
    assert np.abs(Cm - A.reshape(9)).max() < 1e-9 * np.abs(A).max()


@pytest.mark.parametrize("base", [I.BASE_FIXED, I.BASE_SLIP, I.BASE_FREE])
def test_g2p_uniform_field_and_bottom_rule(base):
    """A uniform grid velocity u comes back as v = u with C = 0 at every
    particle (the weights sum to one and their first moment vanishes),
    except that Algorithm 1 zeroes v_z of the bottom-layer particles when the
    base is not free."""
    sc = _scene(g=(0.0, 0.0, 0.0), base=base)
    s = O.make_scene(sc)
    st = _state(sc)
    u = np.array([0.3, -0.2, 0.5])
    nx, ny, nz = sc.gel.nodes
    V = np.tile(u, (nx * ny * nz, 1))
    v, Cm = O.g2p(s, st, V)
    bottom = (st.tag & I.TAG_BOTTOM) != 0
    assert 0 < bottom.sum() < st.n
    ref = np.tile(u, (st.n, 1))
    if base != I.BASE_FREE:
        ref[bottom, 2] = 0.0
    assert np.abs(v - ref).max() < 1e-14
    assert np.abs(Cm).max() < 1e-9 * np.abs(u).max() * 4.0 / sc.gel.dx


# ------------------------------------------------------------------ full steps (Algorithm 1)

def test_free_fall_closed_form():
    """Gravity only, no base or indenter: v_k = k dt g, x_k = x_0 + dt^2 g k(k+1)/2
    (symplectic Euler of Eq. 9; x and F move once per step), F stays I."""
    sc = _scene(base=I.BASE_FREE)
    s = O.make_scene(sc)
    st = _state(sc)
    x0 = st.x.copy()
    ind = O.make_indenter(sc.ind)
    k = 25
    O.run(s, ind, sc.keyframes, 0, k, st)
    g = np.array(sc.mat.gravity)
    dt = sc.solver.dt
    assert np.abs(st.v - k * dt * g).max() < 1e-12
    assert np.abs(st.x - (x0 + dt * dt * g * k * (k + 1) / 2)).max() < 1e-15
    assert np.abs(st.F - np.eye(3).reshape(9)).max() < 1e-12


def test_energy_balance_free_oscillation():
    """A free block given a uniform dilation rate (an affine field, F = I)
    oscillates: kinetic energy (incl. the APIC affine part) turns into
    Neo-Hookean energy and back.  The total may only decay (transfer
    dissipation at the free surface), never grow; a wrong scale or sign of
    the stress impulse of Eq. 4 makes it grow or blow up."""
    n = 16
    dx = 8e-3 / n
    sc = _scene(cx=n, cy=n, cz=n, dx=dx, E=1.5e5, nu=0.3, g=(0.0, 0.0, 0.0),
                base=I.BASE_FREE, dt=2.5e-6)
    s = O.make_scene(sc)
    st = _state(sc)
    A = 3.0
    st.v[:] = A * (st.x - st.x.mean(0))
    st.C[:] = (A * np.eye(3)).reshape(9)
    mu, lam = O.lame(sc.mat.E, sc.mat.nu)
    V0 = dx ** 3 / 8
    mp = sc.mat.rho * V0
    ind = O.make_indenter(sc.ind)

    def energy():
        Fm = st.F.reshape(-1, 3, 3)
        J = np.linalg.det(Fm)
        psi = 0.5 * mu * (np.einsum("pab,pab->p", Fm, Fm) - 3) - mu * np.log(J) + 0.5 * lam * np.log(J) ** 2
        ke = 0.5 * mp * (st.v ** 2).sum() + 0.5 * mp * dx * dx / 4 * (st.C ** 2).sum()
        return ke, V0 * psi.sum()

    ke0, pe0 = energy()
    e0 = ke0 + pe0
    peak_pe = 0.0
    for blk in range(4):
        O.run(s, ind, sc.keyframes, blk * 40, 40, st)
        ke, pe = energy()
        peak_pe = max(peak_pe, pe / e0)
        assert (ke + pe) / e0 < 1.01, (blk, ke, pe, e0)
        assert (ke + pe) / e0 > 0.9, (blk, ke, pe, e0)
    assert peak_pe > 0.7


@pytest.mark.parametrize("base", [I.BASE_FIXED, I.BASE_SLIP, I.BASE_FREE])
def test_grid_update_boundary_rules(base):
    """Eq. 5 and the boundary rules on a grid with known momenta: a node with
    mass gets V = MG / M + dt g; a massless node stays at rest; the two-node
    padding ring at -x, +x, -y, +y and +z is held at rest; nodes at or below
    the gel base (physical z index <= 0) are held at rest (fixed base), lose
    only their normal component (slip base) or keep their velocity (free).
    A ring one node too wide or narrow, a base plane one node off or a
    swapped axis fails this."""
    sc = _scene(cx=8, cy=12, cz=4, g=(0.0, 0.0, -9.81), base=base)
    s = O.make_scene(sc)
    nx, ny, nz = sc.gel.nodes
    assert nx != ny                                   # so that swapped axes show
    ox, oy, oz = sc.gel.origin
    nn = nx * ny * nz
    rng = np.random.default_rng(9)
    M = rng.uniform(0.5, 2.0, nn)
    M[rng.random(nn) < 0.1] = 0.0                      # some empty nodes
    u = rng.standard_normal((nn, 3))
    V, cnt = O.grid_update(s, O.make_indenter(I.no_indenter()), O.pose(sc.keyframes, 0, s.dt, 0.0),
                           M, M[:, None] * u)
    assert cnt == 0
    az, ay, ax = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    az, ay, ax = az.ravel(), ay.ravel(), ax.ravel()
    ref = np.where(M[:, None] > 0, u + s.dt * np.array([0.0, 0.0, -9.81]), 0.0)
    ring = (ax < 2) | (ay < 2) | (ax >= nx - 2) | (ay >= ny - 2) | (az >= nz - 2)
    ref[ring] = 0.0
    low = (az - oz <= 0) & ~ring
    if base == I.BASE_FIXED:
        ref[low] = 0.0
    elif base == I.BASE_SLIP:
        ref[low, 2] = 0.0
    assert low.sum() > 0 and ring.sum() > 0 and (~ring & ~low & (M > 0)).sum() > 0
    assert np.abs(V - ref).max() <= 1e-15 * np.abs(ref).max() + 1e-300


def test_uniaxial_compression_linear_elasticity():
    """Block on a frictionless base pressed slowly by a frictionless plate to
    strain 1e-3: interior stress is uniaxial, sigma_zz = E eps_zz (2%) and the
    lateral strain is -nu eps_zz (5%)."""
    dx, cz = 1e-3, 8
    gel = I.Gel(8, 8, cz, dx, seed=11)
    H = gel.height
    plate = I.box(20e-3, 20e-3, 5e-3, 0.5e-3, 0.0)
    nramp, nhold = 500, 300
    d = 1e-3 * H
    kf = I.keyframes([(0, 4e-3, 4e-3, H, 0.0), (nramp, 4e-3, 4e-3, H - d, 0.0)])
    E, nu = 1.5e5, 0.45
    sc = I.Scene(gel, I.Material(E=E, nu=nu, gravity=(0.0, 0.0, 0.0)), plate, kf,
                 I.Solver(dt=1.5e-5, relrest_limit=1, base_mode=I.BASE_SLIP))
    s = O.make_scene(sc)
    ind = O.make_indenter(plate)
    st = _state(sc)
    O.run(s, ind, kf, 0, nramp, st)
    x0 = np.asarray(I.gel_particles(gel)[0], dtype=np.float64)
    inner = ((x0[:, 0] > 2 * dx) & (x0[:, 0] < 6 * dx) & (x0[:, 1] > 2 * dx) & (x0[:, 1] < 6 * dx)
             & (x0[:, 2] > 2 * dx) & (x0[:, 2] < 6 * dx))
    mu, lam = O.lame(E, nu)
    acc = []
    for blk in range(nhold // 20):
        O.run(s, ind, kf, nramp + blk * 20, 20, st)
        Fm = st.F.reshape(-1, 3, 3)[inner]
        J = np.linalg.det(Fm)
        sig = np.array([O.kirchhoff(f, mu, lam) for f in Fm]) / J[:, None, None]
        acc.append((Fm[:, 2, 2].mean() - 1, 0.5 * (Fm[:, 0, 0].mean() + Fm[:, 1, 1].mean()) - 1,
                    sig[:, 2, 2].mean(), 0.5 * (sig[:, 0, 0].mean() + sig[:, 1, 1].mean())))
    ezz, exx, szz, sxx = np.mean(np.array(acc), axis=0)
    assert ezz < -5e-4
    assert abs(szz - E * ezz) < 0.02 * abs(E * ezz), (szz, E * ezz)
    assert abs(exx + nu * ezz) < 0.05 * abs(nu * ezz), (exx, -nu * ezz)
    assert abs(sxx) < 0.05 * abs(szz)


# ------------------------------------------------------------------ indenter geometry

def _fd_grad(ind, q, h=1e-7):
    g = np.zeros(3)
    for a in range(3):
        e = np.zeros(3); e[a] = h
        g[a] = (O.sdf_local(ind, q + e)[0] - O.sdf_local(ind, q - e)[0]) / (2 * h)
    return g


@pytest.mark.parametrize("ind", [I.sphere(4e-3, 0.5), I.cylinder(3e-3, 10e-3, 0.25e-3, 0.5),
                                 I.box(3e-3, 2e-3, 1.5e-3, 0.25e-3, 0.5),
                                 I.prism(6e-3, 10e-3, 0.25e-3, 0.5)])
def test_sdf_eikonal_and_gradient(ind):
    """Exact SDFs: |grad phi| = 1 and the analytic gradient equals central
    differences of phi (away from the medial axis)."""
    o = O.make_indenter(ind)
    n_ok = 0
    for q in RNG.uniform(-8e-3, 8e-3, (400, 3)):
        phi, g = O.sdf_local(o, q)
        if phi < -0.2e-3 and ind.kind != I.SPHERE:
            continue                       # interior medial axes: gradient kinks
        gf = _fd_grad(o, q)
        assert abs(np.linalg.norm(g) - 1) < 1e-9
        assert np.abs(g - gf).max() < 1e-4, (q, g, gf)
        n_ok += 1
    assert n_ok > 100


def test_sdf_surface_points_and_tip():
    s3 = math.sqrt(3.0)
    sp = O.make_indenter(I.sphere(4e-3, 0.5))
    for u in RNG.standard_normal((20, 3)):
        u /= np.linalg.norm(u)
        assert abs(O.sdf_local(sp, 4e-3 * u)[0]) < 1e-15
    cy = O.make_indenter(I.cylinder(3e-3, 10e-3, 0.25e-3, 0.5))
    assert abs(O.sdf_local(cy, [0, 0, -5e-3])[0]) < 1e-15          # flat face
    assert abs(O.sdf_local(cy, [3e-3, 0, 0])[0]) < 1e-15           # side
    bx = O.make_indenter(I.box(3e-3, 2e-3, 1.5e-3, 0.25e-3, 0.5))
    assert abs(O.sdf_local(bx, [0, 0, -1.5e-3])[0]) < 1e-15
    assert abs(O.sdf_local(bx, [3e-3, 0.5e-3, 0])[0]) < 1e-15
    pr = I.prism(6e-3, 10e-3, 0.25e-3, 0.5)
    po = O.make_indenter(pr)
    inr = 6e-3 / (2 * s3)
    assert abs(O.sdf_local(po, [0, 0, inr])[0]) < 1e-15            # top face
    assert abs(O.sdf_local(po, [0, 0, -pr.tip_offset])[0]) < 1e-15  # rounded apex = tip
    # every tip offset puts the lowest point of the shape at the tip
    for ind in [I.sphere(4e-3, 0.5), I.cylinder(3e-3, 10e-3, 0.25e-3, 0.5),
                I.box(3e-3, 2e-3, 1.5e-3, 0.25e-3, 0.5), pr]:
        o = O.make_indenter(ind)
        assert abs(O.sdf_local(o, [0, 0, -ind.tip_offset])[0]) < 1e-15


def test_perlin_noise_properties():
    """Improved noise vanishes on the integer lattice, so the Perlin plate
    equals the rounded box there; its analytic gradient matches differences."""
    ind = I.perlin_plate(4e-3, 4e-3, 1e-3, 0.25e-3, 0.3e-3, 4e-3, 0.5, 4, 0.5, seed=3)
    o = O.make_indenter(ind)
    bx = O.make_indenter(I.box(4e-3, 4e-3, 1e-3, 0.25e-3, 0.5))
    for a in range(-1, 2):
        for b in range(-1, 2):
            q = np.array([a * 4e-3, b * 4e-3, -2e-3])
            assert abs(O.sdf_local(o, q)[0] - O.sdf_local(bx, q)[0]) < 1e-15
    for q in RNG.uniform(-3.5e-3, 3.5e-3, (100, 3)):
        q[2] = RNG.uniform(-2e-3, -1.2e-3)
        phi, g = O.sdf_local(o, q)
        gf = _fd_grad(o, q, 1e-8)
        gf /= np.linalg.norm(gf)
        assert np.abs(g - gf).max() < 1e-5


def test_world_frame_rotation():
    ind = O.make_indenter(I.box(3e-3, 1e-3, 1e-3, 0.1e-3, 0.5))
    kf = I.keyframes([(0, 1e-3, 2e-3, 3e-3, 0.0), (10, 1e-3, 2e-3, 3e-3, math.pi / 2)])
    ps = O.pose(kf, 10, 1e-5, 1e-3)
    # rotated by 90 deg: the long axis is now along y
    # (keyframe yaw is float32: pi/2 is off by ~4e-8 rad -> ~1e-10 m at 3 mm)
    c = np.array([1e-3, 2e-3, 4e-3])
    assert abs(O.sdf(ind, ps, c + [0, 3e-3, 0])[0]) < 1e-9
    assert abs(O.sdf(ind, ps, c + [1e-3, 0, 0])[0]) < 1e-9
    phi, n = O.sdf(ind, ps, c + [0, 4e-3, 0])
    assert abs(phi - 1e-3) < 1e-9 and abs(n[1] - 1) < 1e-9


# ------------------------------------------------------------------ contact, pose, calibration

def _one_node(sc, V_in, node):
    s = O.make_scene(sc)
    nn = O.n_nodes(s)
    M = np.zeros(nn)
    MG = np.zeros((nn, 3))
    M[node] = 2.0
    MG[node] = 2.0 * np.asarray(V_in)
    return s, M, MG


def test_contact_projection_invariants():
    """Stick: V = v_obj; frictionless: only the approaching normal part is
    removed; separating and outside nodes keep their velocity."""
    dx = 1e-3
    gel = I.Gel(8, 8, 4, dx)
    nx, ny, nz = gel.nodes
    ox, oy, oz = gel.origin
    ai, aj, ak = ox + 4, oy + 4, oz + 3
    node = (ak * ny + aj) * nx + ai
    xw = np.array([4 * dx, 4 * dx, 3 * dx])
    kf = I.keyframes([(0, 4e-3, 4e-3, 2.5e-3, 0.0), (100, 5e-3, 4e-3, 2.5e-3, 0.5)])
    for mu in (1e30, 0.0, 0.3):
        ind = I.sphere(2e-3, mu)
        sc = I.Scene(gel, I.Material(gravity=(0.0, 0.0, 0.0)), ind, kf, I.Solver(dt=1e-5))
        o = O.make_indenter(ind)
        ps = O.pose(kf, 10, 1e-5, ind.tip_offset)
        phi, n = O.sdf(o, ps, xw)
        assert phi < 0
        vo = np.array([ps.vlin[0] - ps.omega * (xw[1] - ps.c[1]),
                       ps.vlin[1] + ps.omega * (xw[0] - ps.c[0]), ps.vlin[2]])
        V_in = vo - 0.05 * n + np.array([0.02, -0.01, 0.0])     # approaching
        s, M, MG = _one_node(sc, V_in, node)
        V, cnt = O.grid_update(s, o, ps, M, MG)
        assert cnt == 1
        if mu > 1e20:
            assert np.abs(V[node] - vo).max() < 1e-14
        elif mu == 0.0:
            vr_in, vr = V_in - vo, V[node] - vo
            assert abs(vr @ n) < 1e-15                              # no normal approach left
            t_in, t = vr_in - (vr_in @ n) * n, vr - (vr @ n) * n
            assert np.abs(t - t_in).max() < 1e-15                   # tangential untouched
        else:
            vr_in, vr = V_in - vo, V[node] - vo
            t_in = vr_in - (vr_in @ n) * n
            vn = vr_in @ n
            assert np.linalg.norm(vr) == pytest.approx(max(0.0, np.linalg.norm(t_in) + mu * vn), rel=1e-12)
        V_sep = vo + 0.05 * n                                       # separating
        s, M, MG = _one_node(sc, V_sep, node)
        V, cnt = O.grid_update(s, o, ps, M, MG)
        assert cnt == 0 and np.abs(V[node] - V_sep).max() < 1e-15


def test_static_kinetic_friction_projection():
    """A kinetic coefficient mu_k < mu (the long-slide reading of Sec. VI):
    a node sticks while |v_t| <= mu |v_n|, and once it slips its tangential
    relative speed drops by mu_k |v_n|.  Hand-worked with v_n = -0.05 m/s,
    mu = 0.5, mu_k = 0.3: |v_t| = 0.02 sticks (it would slip under mu_k
    alone), |v_t| = 0.04 leaves 0.04 - 0.015 = 0.025 along v_t, and with mu_k
    unset the same node keeps 0.04 - 0.025 = 0.015."""
    dx = 1e-3
    gel = I.Gel(8, 8, 4, dx)
    nx, ny, nz = gel.nodes
    ox, oy, oz = gel.origin
    node = ((oz + 3) * ny + oy + 4) * nx + ox + 4
    xw = np.array([4 * dx, 4 * dx, 3 * dx])
    kf = I.keyframes([(0, 4e-3, 4e-3, 2.5e-3, 0.0), (100, 5e-3, 4e-3, 2.5e-3, 0.5)])
    for mu_k, t_len, want in ((0.3, 0.02, 0.0), (0.3, 0.04, 0.025), (0.0, 0.04, 0.015)):
        ind = I.sphere(2e-3, 0.5)
        ind.mu_k = mu_k
        sc = I.Scene(gel, I.Material(gravity=(0.0, 0.0, 0.0)), ind, kf, I.Solver(dt=1e-5))
        o = O.make_indenter(ind)
        ps = O.pose(kf, 10, 1e-5, ind.tip_offset)
        phi, n = O.sdf(o, ps, xw)
        assert phi < 0
        vo = np.array([ps.vlin[0] - ps.omega * (xw[1] - ps.c[1]),
                       ps.vlin[1] + ps.omega * (xw[0] - ps.c[0]), ps.vlin[2]])
        t_hat = np.cross(n, [1.0, 0.0, 0.0])
        t_hat /= np.linalg.norm(t_hat)
        s, M, MG = _one_node(sc, vo - 0.05 * n + t_len * t_hat, node)
        V, cnt = O.grid_update(s, o, ps, M, MG)
        assert cnt == 1
        vr = V[node] - vo
        assert abs(vr @ n) < 1e-15
        assert np.abs(vr - want * t_hat).max() < 1e-15


def test_object_particle_p2g_transfers_the_rigid_motion_exactly():
    """Object particles (the paper's particle-represented indenter) carry
    the rigid velocity v_lin + omega z x (x - c) and its affine field, so
    their P2G alone gives every node with mass exactly the rigid velocity at
    the node (APIC transfers affine fields exactly), the total mass n m and
    the total momentum m sum v.  A wrong sign of C or of the rotation, or a
    missing affine term, fails this."""
    dx = 0.5e-3
    gel = I.Gel(16, 16, 8, dx)
    # the sphere and its stencils stay inside the node box (z up to 7.5 mm)
    kf = I.keyframes([(0, 4e-3, 4e-3, 4.4e-3, 0.0), (100, 4.6e-3, 3.7e-3, 4.2e-3, 0.4)])
    ind = I.sphere(1e-3, 0.5)
    ind.obj = I.object_particles(ind, dx / 2)
    ind.obj_m = 2.5e-8
    sc = I.Scene(gel, I.Material(gravity=(0.0, 0.0, 0.0)), ind, kf, I.Solver(dt=1e-5))
    s, o = O.make_scene(sc), O.make_indenter(ind)
    ps = O.pose(kf, 37, 1e-5, ind.tip_offset)
    assert abs(ps.omega) > 0 and abs(ps.vlin[0]) > 0
    M, MG = O.object_p2g(s, o, ps)
    n = len(ind.obj)
    assert M.sum() == pytest.approx(n * ind.obj_m, rel=1e-12)
    q = ind.obj.astype(np.float64)
    xw = np.stack([ps.c[0] + ps.cs * q[:, 0] - ps.sn * q[:, 1], ps.c[1] + ps.sn * q[:, 0] + ps.cs * q[:, 1],
                   ps.c[2] + q[:, 2]], 1)
    vq = np.stack([ps.vlin[0] - ps.omega * (xw[:, 1] - ps.c[1]), ps.vlin[1] + ps.omega * (xw[:, 0] - ps.c[0]),
                   np.full(n, ps.vlin[2])], 1)
    assert np.abs(MG.sum(0) - ind.obj_m * vq.sum(0)).max() < 1e-12 * ind.obj_m * n
    nx, ny, nz = gel.nodes
    ox, oy, oz = gel.origin
    idx = np.nonzero(M > 0)[0]
    ax, ay, az = idx % nx, (idx // nx) % ny, idx // (nx * ny)
    xn = np.stack([(ax - ox) * dx, (ay - oy) * dx, (az - oz) * dx], 1)
    vn = np.stack([ps.vlin[0] - ps.omega * (xn[:, 1] - ps.c[1]), ps.vlin[1] + ps.omega * (xn[:, 0] - ps.c[0]),
                   np.full(idx.size, ps.vlin[2])], 1)
    assert np.abs(MG[idx] / M[idx, None] - vn).max() < 1e-12


def test_object_particles_press_the_gel():
    """A press with the particle-represented sphere (no SDF contact) pushes
    the gel top under it down, by an amount comparable to the SDF contact
    press of the same trajectory, and a pure press still takes one pass per
    substep."""
    sc = I.scene_small(cx=12, cy=12, cz=4, n_press=60, mu=0.6, press=0.4e-3)
    out = {}
    for mode, scn in (("sdf", sc), ("particles", I.with_object_particles(sc))):
        s, o = O.make_scene(scn), O.make_indenter(scn.ind)
        st = _state(scn)
        z0 = st.x[:, 2].copy()
        p, _ = O.run(s, o, scn.keyframes, 0, 60, st)
        assert np.all(p == 1)
        tip = scn.keyframes[1, 1:3]
        r = np.hypot(st.x[:, 0] - tip[0], st.x[:, 1] - tip[1])
        top = z0 > z0.max() - scn.gel.dx
        out[mode] = (z0 - st.x[:, 2])[top & (r < scn.gel.dx)].mean()
    assert out["particles"] > 0.3 * out["sdf"] > 0, out


def test_pose_interpolation():
    kf = I.keyframes([(0, 0.01, 0.01, 0.005, 0.0), (100, 0.01, 0.01, 0.004, 0.0),
                      (300, 0.013, 0.01, 0.004, 0.0), (500, 0.013, 0.01, 0.004, 0.6)])
    dt = 5e-6
    p = O.pose(kf, 50, dt, 0.002)           # keyframe values are float32-rounded inputs
    assert p.tip[2] == pytest.approx(0.5 * (kf[0, 3] + kf[1, 3]), abs=1e-15)
    assert p.vlin[2] * 100 * dt == pytest.approx(kf[1, 3] - kf[0, 3], rel=1e-12)
    assert p.c[2] == pytest.approx(p.tip[2] + 0.002, abs=1e-15)
    p = O.pose(kf, 200, dt, 0.0)
    assert p.tip[0] == pytest.approx(0.5 * (kf[1, 1] + kf[2, 1]), abs=1e-15)
    p = O.pose(kf, 400, dt, 0.0)
    assert p.yaw == pytest.approx(0.5 * kf[3, 4], rel=1e-15) and p.omega * 200 * dt == pytest.approx(kf[3, 4], rel=1e-12)
    p = O.pose(kf, 9999, dt, 0.0)
    assert p.omega == 0.0 and p.vlin[0] == 0.0 and p.yaw == pytest.approx(kf[3, 4])


def test_nearest_is_argmin():
    x = RNG.uniform(0, 1e-2, (5000, 3))
    xo = np.array([5e-3, 5e-3, 9e-3])
    assert O.nearest(x, xo) == int(np.argmin(((x - xo) ** 2).sum(1)))
    x[17] = x[3]                                        # ties go to the lowest index
    assert O.nearest(x, x[3]) == 3


def test_pure_press_takes_one_pass():
    """No tangential object motion: the relative-rest check accepts the first
    pass, so IMPM equals plain MPM (LIMIT = 1) exactly."""
    sc = I.scene_small(cx=12, cy=12, cz=4, n_press=30)
    s = O.make_scene(sc)
    ind = O.make_indenter(sc.ind)
    a = _state(sc)
    b = a.copy()
    pa, _ = O.run(s, ind, sc.keyframes, 0, 30, a)
    s1 = O.make_scene(sc)
    s1.limit = 1
    pb, _ = O.run(s1, ind, sc.keyframes, 0, 30, b)
    assert np.all(pa == 1) and np.all(pb == 1)
    assert np.array_equal(a.x, b.x) and np.array_equal(a.F, b.F)


def test_sticky_slip_needs_extra_passes():
    """Sliding with friction: the gel surface lags the object, so some steps
    need repeated passes, each bringing the calibration particle closer."""
    sc = I.scene_small(cx=12, cy=12, cz=4, n_press=20, slip=0.5e-3, n_slip=20, mu=1.0, press=0.4e-3)
    s = O.make_scene(sc)
    ind = O.make_indenter(sc.ind)
    st = _state(sc)
    pl, el = O.run(s, ind, sc.keyframes, 0, 40, st)
    assert np.all(pl[:20] == 1)
    assert pl[20:].max() > 1


def _check_pose(c, vlin=(0.0, 0.0, 0.0), omega=0.0):
    """A pose at yaw 0 whose SDF centre is c (the sphere's tip below it)."""
    ps = O.Pose()
    for a in range(3):
        ps.c[a] = c[a]
        ps.tip[a] = c[a]
        ps.vlin[a] = vlin[a]
    ps.yaw, ps.cs, ps.sn, ps.omega = 0.0, 1.0, 0.0, omega
    return ps


def _check_setup(threshold=0.5):
    dx, R = 0.5e-3, 2e-3
    sc = _scene(dx=dx)
    s = O.make_scene(sc)
    s.threshold = threshold
    ind = O.make_indenter(I.sphere(R, 0.5))
    c = np.array([10e-3, 10e-3, 7e-3])
    return s, ind, c, dx, R


def test_relrest_check_hand_worked_slip():
    """Algorithm 1's check at x_e during a slip (v_o = v_lin = 0.1 m/s along
    x, x_e inside the sphere): the tangential mismatch |v_e,t - v_o,t| is
    compared with threshold (0.5) x |v_o,t| -- the object's tangential speed,
    not the particle's -- and the vertical components play no part.  Worked
    by hand: a mismatch of 0.45 |v_o,t| accepts and 0.55 rejects, whichever
    direction it points; v_e,t = 0.6 v_o,t (mismatch 0.4) accepts although
    0.4 > 0.5 x |v_e,t|, and v_e,t = 1.6 v_o,t (mismatch 0.6) rejects
    although 0.6 <= 0.5 x |v_e,t|."""
    s, ind, c, dx, R = _check_setup()
    vo = np.array([0.1, 0.0, 0.0])
    ps = _check_pose(c, vlin=vo)
    xe = c + np.array([0.0, 0.0, -(R - 0.1 * dx)])          # phi = -0.1 dx: in contact
    assert O.sdf(ind, ps, xe)[0] == pytest.approx(-0.1 * dx, abs=1e-12)
    for u in ([1.0, 0.0], [0.0, 1.0], [-0.6, 0.8]):
        u = np.array(u + [0.0])
        assert O.relrest_accept(s, ind, ps, xe, vo + 0.045 * u)
        assert not O.relrest_accept(s, ind, ps, xe, vo + 0.055 * u)
    assert O.relrest_accept(s, ind, ps, xe, [0.06, 0.0, 0.0])
    assert not O.relrest_accept(s, ind, ps, xe, [0.16, 0.0, 0.0])
    assert O.relrest_accept(s, ind, ps, xe, [0.11, 0.0, 5.0])      # v_z is not compared
    assert O.relrest_accept(s, ind, ps, xe, [0.1, 0.0, -5.0])
    # the threshold scales the bound: at 0.4 the 0.45 mismatch rejects
    s4, _, _, _, _ = _check_setup(threshold=0.4)
    assert not O.relrest_accept(s4, ind, ps, xe, vo + [0.045, 0.0, 0.0])
    assert O.relrest_accept(s4, ind, ps, xe, vo + [0.035, 0.0, 0.0])


def test_relrest_check_hand_worked_rotation():
    """During a turn (v_lin = 0, omega = 2 rad/s about the vertical axis
    through the centre) the object velocity at x_e = c + (r, 0, .) is
    omega z x (x_e - c) = (0, omega r, 0): a particle moving with it accepts,
    one moving the opposite way (mismatch 2 omega r) or not at all (mismatch
    omega r > 0.5 omega r) rejects."""
    s, ind, c, dx, R = _check_setup()
    om, r = 2.0, 1.5e-3
    ps = _check_pose(c, omega=om)
    xe = c + np.array([r, 0.0, -np.sqrt(R ** 2 - r ** 2) + 0.2 * dx])
    assert O.sdf(ind, ps, xe)[0] < 0.0
    assert O.relrest_accept(s, ind, ps, xe, [0.0, om * r, 0.0])
    assert O.relrest_accept(s, ind, ps, xe, [0.3 * om * r, 0.8 * om * r, 0.0])   # mismatch 0.36 omega r
    assert not O.relrest_accept(s, ind, ps, xe, [0.0, -om * r, 0.0])
    assert not O.relrest_accept(s, ind, ps, xe, [0.0, 0.0, 0.0])
    assert not O.relrest_accept(s, ind, ps, xe, [om * r, 0.0, 0.0])          # right speed, wrong direction


def test_relrest_check_accepts_out_of_contact_and_without_tangential_motion():
    """The two early accepts of the reading of Algorithm 1: x_e more than one
    cell away from the object (phi(x_e) > dx), and an object with no
    tangential velocity at x_e (|v_o,t| < 1e-6 m/s, a pure press); just
    inside those bounds the same mismatched particle rejects."""
    s, ind, c, dx, R = _check_setup()
    ps = _check_pose(c, vlin=(0.1, 0.0, 0.0))
    for gap, ok in ((1.5, True), (1.05, True), (0.9, False), (0.0, False)):
        xe = c + np.array([0.0, 0.0, -(R + gap * dx)])
        assert O.sdf(ind, ps, xe)[0] == pytest.approx(gap * dx, abs=1e-12)
        assert O.relrest_accept(s, ind, ps, xe, [0.0, 0.0, 0.0]) is ok, gap
    xe = c + np.array([0.0, 0.0, -(R - 0.1 * dx)])
    press = _check_pose(c, vlin=(0.0, 0.0, -0.05))
    assert O.relrest_accept(s, ind, press, xe, [0.3, 0.2, 0.0])
    assert O.relrest_accept(s, ind, _check_pose(c, vlin=(5e-7, 0.0, -0.05)), xe, [0.3, 0.2, 0.0])
    assert not O.relrest_accept(s, ind, _check_pose(c, vlin=(2e-6, 0.0, -0.05)), xe, [0.3, 0.2, 0.0])
    none = O.make_indenter(I.no_indenter())
    assert O.relrest_accept(s, none, ps, xe, [0.3, 0.2, 0.0])


@pytest.mark.parametrize("threads", [3, 4])
def test_all_cores_oracle_equals_serial(threads):
    """The all-cores variant (run_par: particle chunks P2G'd into private
    grids summed in chunk order) differs from the serial oracle only in the
    order of the grid sums: through a sticking slip with repeated passes the
    pass counts and calibration particles are the same and the states agree
    to 1e-12 relative."""
    sc = I.scene_small(cx=12, cy=12, cz=4, n_press=20, slip=0.5e-3, n_slip=20, mu=1.0, press=0.4e-3)
    s = O.make_scene(sc)
    ind = O.make_indenter(sc.ind)
    a = _state(sc)
    b = a.copy()
    pa, ea = O.run(s, ind, sc.keyframes, 0, 40, a)
    pb, eb = O.run_par(s, ind, sc.keyframes, 0, 40, b, threads)
    assert pa.max() > 1
    assert np.array_equal(pa, pb) and np.array_equal(ea, eb)
    for u, w in ((a.x, b.x), (a.v, b.v), (a.C, b.C), (a.F, b.F)):
        assert np.linalg.norm(u - w) <= 1e-12 * np.linalg.norm(u)


def test_all_cores_oracle_equals_serial_with_object_particles():
    """The same with the particle-represented indenter, whose P2G the
    all-cores variant adds after summing the private grids."""
    sc = I.with_object_particles(I.scene_small(cx=12, cy=12, cz=4, n_press=20, slip=0.3e-3, n_slip=20, mu=0.6,
                                               press=0.4e-3))
    s = O.make_scene(sc)
    ind = O.make_indenter(sc.ind)
    a = _state(sc)
    b = a.copy()
    pa, ea = O.run(s, ind, sc.keyframes, 0, 40, a)
    pb, eb = O.run_par(s, ind, sc.keyframes, 0, 40, b, 4)
    assert np.array_equal(pa, pb) and np.array_equal(ea, eb)
    for u, w in ((a.x, b.x), (a.v, b.v), (a.F, b.F)):
        assert np.linalg.norm(u - w) <= 1e-12 * np.linalg.norm(u)
    assert (_state(sc).x[:, 2] - a.x[:, 2]).max() > 0.1 * sc.gel.dx          # it pressed


def test_frictionless_sphere_rotation_invariance():
    """A frictionless sphere spinning about its vertical axis exerts no
    tangential force (plain MPM): the surface field is unchanged."""
    sc = I.scene_small(cx=12, cy=12, cz=4, n_press=20, rotate=0.8, n_rot=20, mu=0.0, limit=1)
    s = O.make_scene(sc)
    ind = O.make_indenter(sc.ind)
    a = _state(sc)
    b = a.copy()
    O.run(s, ind, sc.keyframes, 0, 40, a)
    kf_hold = sc.keyframes[:2]
    O.run(s, ind, kf_hold, 0, 40, b)
    assert np.abs(a.x - b.x).max() < 1e-15
    assert a.x[:, 2].min() < sc.gel.height - 0.3 * sc.gel.dx    # it did press


def _drag_run(mu, slip=0.0, rotate=0.0, n_move=0, mu_k=0.0):
    """Press 0.4 mm in 60 substeps, then slip along +x or turn about the
    vertical axis in n_move substeps; returns the top-layer particles within
    the contact patch at the end of the press (before, after) and the tip."""
    sc = I.scene_small(cx=12, cy=12, cz=4, n_press=60, slip=slip, n_slip=n_move if slip else 0, rotate=rotate,
                       n_rot=n_move if rotate else 0, mu=mu, press=0.4e-3)
    sc.ind.mu_k = mu_k
    s = O.make_scene(sc)
    ind = O.make_indenter(sc.ind)
    st = _state(sc)
    O.run(s, ind, sc.keyframes, 0, 60, st)
    x1 = st.x.copy()
    O.run(s, ind, sc.keyframes, 60, n_move, st)
    tip = sc.keyframes[1, 1:3]
    dx = sc.gel.dx
    r = np.hypot(x1[:, 0] - tip[0], x1[:, 1] - tip[1])
    return x1, st.x, tip, r, (x1[:, 2] > x1[:, 2].max() - dx), dx


def test_sticking_slip_drags_the_contact_patch():
    """Coulomb friction in the stick regime (relative rest, mu = 1) drags the
    gel under the indenter along the slip direction, by less than the slip
    itself (the elastic gel lags); without friction there is no tangential
    traction and the patch stays nearly in place.  A wrong sign of the
    object velocity or of the tangential projection, or friction that is not
    applied, fails this."""
    slip = 0.5e-3
    out = {}
    for mu in (1.0, 0.0):
        x1, x2, tip, r, top, dx = _drag_run(mu, slip=slip, n_move=100)
        patch = top & (r < 1.5 * dx)
        assert patch.sum() >= 20
        d = (x2 - x1)[patch]
        out[mu] = d[:, 0].mean() / slip
        assert abs(d[:, 1].mean()) < 0.02 * slip          # nothing across the slip direction
    assert 0.2 < out[1.0] < 1.0, out
    assert abs(out[0.0]) < 0.1, out


def test_kinetic_friction_lowers_the_drag_of_a_long_slide():
    """A long slide (1.5 mm, several contact radii) at mu = 1: once the
    contact slips, a lower kinetic coefficient drags the patch less, in
    order of mu_k (measured 0.19, 0.094, 0.020 of the slide for mu_k = 1,
    0.6, 0.3), and never backwards.  A kinetic coefficient that is ignored,
    or that also decides the stick, fails this."""
    slip = 1.5e-3
    drag = []
    for mu_k in (0.0, 0.6, 0.3):
        x1, x2, tip, r, top, dx = _drag_run(1.0, slip=slip, n_move=150, mu_k=mu_k)
        patch = top & (r < 1.5 * dx)
        drag.append((x2 - x1)[patch][:, 0].mean() / slip)
    assert drag[0] > 1.5 * drag[1] > 0 and drag[1] > 2 * drag[2] > 0, drag


@pytest.mark.parametrize("rotate", [0.3, -0.3])
def test_sticking_rotation_turns_the_contact_patch(rotate):
    """A sticking indenter that turns about its vertical axis by theta turns
    the contact patch the same way (omega x r, counter-clockwise for theta >
    0), by a fraction of theta.  The frictionless case is the rotation
    invariance pin above."""
    x1, x2, tip, r, top, dx = _drag_run(1.0, rotate=rotate, n_move=100)
    ring = top & (r > 0.5 * dx) & (r < 2.0 * dx)
    assert ring.sum() >= 40
    a1 = np.arctan2(x1[ring, 1] - tip[1], x1[ring, 0] - tip[0])
    a2 = np.arctan2(x2[ring, 1] - tip[1], x2[ring, 0] - tip[0])
    turn = np.angle(np.exp(1j * (a2 - a1))).mean() / rotate
    assert 0.1 < turn < 1.0, turn


# ------------------------------------------------------------------ surface readout

def test_surface_readout_closed_forms():
    dx = 0.5e-3
    W = 10
    # regular lattice: two particles per pixel and axis, symmetric about centres
    u = (np.arange(2 * W) + 0.5) * dx / 2
    X, Y = np.meshgrid(u, u, indexing="xy")
    a, b, c = 0.07, -0.04, 3e-3
    Z = a * X + b * Y + c
    x = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    tag = np.full(x.shape[0], I.TAG_TOP, dtype=np.uint32)
    st = O.State(x, np.zeros_like(x), np.zeros((x.shape[0], 9)), np.zeros((x.shape[0], 9)), tag)
    h, n = O.surface(st, W, W, dx, 0.0)
    Xc = (np.arange(W) + 0.5) * dx
    inner = slice(1, W - 1)
    href = a * Xc[None, :] + b * Xc[:, None] + c          # h[row=y, col=x]
    assert np.abs(h[inner, inner] - href[inner, inner]).max() < 1e-15
    nref = np.array([-a, -b, 1]) / math.sqrt(1 + a * a + b * b)
    inner2 = slice(2, W - 2)              # central differences reach one pixel further
    assert np.abs(n[inner2, inner2] - nref).max() < 1e-12
    # vertical translation moves h by the same amount everywhere
    st.x[:, 2] += 1e-4
    h2, _ = O.surface(st, W, W, dx, 0.0)
    assert np.abs(h2 - h - 1e-4).max() < 1e-15
    # particles without the top tag are ignored; empty pixels read h_empty
    st.tag[:] = 0
    h3, n3 = O.surface(st, W, W, dx, 7.0)
    assert np.all(h3 == 7.0) and np.all(n3[..., 2] == 1.0)


def _top_lattice(W, dx, z0=3e-3):
    """Two particles per pixel and axis, symmetric about the pixel centres."""
    u = (np.arange(2 * W) + 0.5) * dx / 2
    X, Y = np.meshgrid(u, u, indexing="xy")
    return np.stack([X.ravel(), Y.ravel(), np.full(X.size, z0)], 1)


def test_surface_displacement_closed_forms():
    """The displacement field is a normalised B-spline splat of x - x_ref at
    the reference positions: a rigid translation comes back exactly
    everywhere; a linear field u = A x_ref comes back as A times the pixel
    centre on the interior pixels (the lattice is symmetric about them, so
    the weighted mean reference position is the centre); untagged particles
    are ignored and pixels out of every particle's reach read zero."""
    dx, W = 0.5e-3, 10
    xref = _top_lattice(W, dx)
    n = xref.shape[0]
    tag = np.full(n, I.TAG_TOP, dtype=np.uint32)
    z = np.zeros((n, 9))

    def disp(x, t, xr=xref, Wd=W):
        return O.surface_disp(O.State(x, np.zeros_like(x), z[:len(x)], z[:len(x)], t), xr, Wd, Wd, dx)

    u0 = np.array([3e-5, -2e-5, -7e-5])
    u = disp(xref + u0, tag)
    assert np.abs(u - u0).max() < 1e-18
    A = np.array([[0.01, -0.03, 0.02], [0.04, 0.005, -0.01], [-0.02, 0.03, 0.015]])
    u = disp(xref + xref @ A.T, tag)
    Xc = (np.arange(W) + 0.5) * dx
    ref = np.einsum("ij,yxj->yxi", A, np.stack(np.broadcast_arrays(Xc[None, :], Xc[:, None], 3e-3), -1))
    inner = slice(1, W - 1)
    assert np.abs(u[inner, inner] - ref[inner, inner]).max() < 1e-17
    # untagged particles with a large displacement change nothing
    t2 = tag.copy()
    t2[::3] = 0
    x2 = xref + u0
    x2[::3] += 1e-3
    xr2 = xref.copy()
    u2 = disp(x2, t2)
    assert np.abs(u2 - u0).max() < 1e-18
    # particles only in the left two pixel columns: far pixels read zero
    left = xr2[:, 0] < 2 * dx
    u3 = O.surface_disp(O.State((xref + u0)[left], np.zeros((left.sum(), 3)), z[:left.sum()], z[:left.sum()],
                                tag[left]), xref[left], W, W, dx)
    assert np.all(u3[:, 4:] == 0.0) and np.abs(u3[:, :2] - u0).max() < 1e-18


def test_indenter_height_of_a_sphere():
    """The underside of a sphere of radius R centred at c above the pixel
    column at distance rho from its axis lies at c_z - sqrt(R^2 - rho^2):
    the height map reads that minus the gel top, +clip where the column
    misses the sphere, clipped to [-clip, clip]; turning the sphere about
    its axis changes nothing."""
    Hgel, R, pitch, W, clip = 4e-3, 2e-3, 0.5e-3, 20, 3e-3
    ind = O.make_indenter(I.sphere(R, 0.5))
    tip = np.array([5.1e-3, 4.9e-3, Hgel - 0.2e-3])          # pressed 0.2 mm into the gel
    for yaw in (0.0, 0.7):
        kf = I.keyframes([(0, tip[0], tip[1], tip[2], yaw)])
        ps = O.pose(kf, 0, 1e-5, R)
        h = O.indenter_height(ind, ps, Hgel, W, W, pitch, clip, 0.05e-3)
        xc = (np.arange(W) + 0.5) * pitch
        rho2 = (xc[None, :] - kf[0, 1]) ** 2 + (xc[:, None] - kf[0, 2]) ** 2
        inside = rho2 < R * R
        ref = np.where(inside, kf[0, 3] + R - np.sqrt(np.where(inside, R * R - rho2, 0.0)) - Hgel, clip)
        ref = np.clip(ref, -clip, clip)
        away = np.abs(np.sqrt(rho2) - R) > 1e-5                  # the scan step can miss a sliver at the rim
        assert inside.sum() > 40 and (~inside).sum() > 40
        assert np.abs(h - ref)[away].max() < 1e-12
        assert h.min() < 0.0                                     # the pressed centre is below the gel top
