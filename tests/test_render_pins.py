"""Pins of the sensor-image oracle (oracle/render_oracle.c): the path tracer
against Lambert's polygon irradiance and exact structural properties, and
the image metrics against closed forms.  CPU only."""
import math

import numpy as np
import pytest

from oracle import render_oracle as RO

PITCH = 1e-3


def _flat(W=4, H=4, z=5e-3):
    return np.full((H, W), z)


def _panel_below(z_s):
    """One upward-emitting 2 x 2 mm panel 2 mm below the surface."""
    return [((2e-3, 2e-3, z_s - 2e-3), (1e-3, 0.0, 0.0), (0.0, 1e-3, 0.0), (1.0, 1.0, 1.0))]


def _lambert_irradiance(P, N, verts):
    """Irradiance at P (unit normal N) from a unit-radiance polygon, by
    Lambert's formula: (1/2) sum over edges of the edge's angle times the
    normal component of the unit normal of the plane through P and the edge."""
    E = 0.0
    r = [(np.asarray(v) - P) / np.linalg.norm(np.asarray(v) - P) for v in verts]
    for k in range(len(r)):
        a, b = r[k], r[(k + 1) % len(r)]
        g = np.cross(a, b)
        E += math.acos(np.clip(a @ b, -1, 1)) * (g / np.linalg.norm(g)) @ N
    return 0.5 * abs(E)


def test_one_bounce_flat_surface_matches_lambert_irradiance():
    """A flat membrane (albedo 0.7) over one Lambertian panel: the pixel
    value of a single reflection is albedo E / pi, E from Lambert's formula
    at the pixel's hit points; 4096 samples per pixel, within 4 standard
    errors of the hit fraction."""
    z = 5e-3
    h = _flat(z=z)
    spp = 4096
    d = RO.make_desc(_panel_below(z), spp, 1, 0.0, 12345)
    img = RO.render(h, 0.7, PITCH, d)
    c = np.array([2e-3, 2e-3, z - 2e-3])
    verts = [c + np.array(o) for o in ((-1e-3, -1e-3, 0), (1e-3, -1e-3, 0), (1e-3, 1e-3, 0), (-1e-3, 1e-3, 0))]
    N = np.array([0.0, 0.0, -1.0])
    for i in range(4):
        for j in range(4):
            # the pixel averages hit points over its area: integrate E over a 16 x 16 sub-grid
            xs = (j + (np.arange(16) + 0.5) / 16) * PITCH
            ys = (i + (np.arange(16) + 0.5) / 16) * PITCH
            E = np.mean([_lambert_irradiance(np.array([x, y, z]), N, verts) for y in ys for x in xs])
            p = E / math.pi
            se = math.sqrt(p * (1 - p) / spp)
            assert abs(img[i, j, 0] / 0.7 - p) < 4 * se + 1e-12, (i, j, img[i, j, 0] / 0.7, p, se)
            assert img[i, j, 0] == img[i, j, 1] == img[i, j, 2]


def test_dark_inputs_give_black():
    h = _flat()
    d = RO.make_desc(_panel_below(5e-3), 64, 3, 0.0, 1)
    assert np.all(RO.render(h, 0.0, PITCH, d) == 0.0)
    d0 = RO.make_desc([(c, u, v, (0.0, 0.0, 0.0)) for c, u, v, _ in _panel_below(5e-3)], 64, 3, 0.0, 1)
    assert np.all(RO.render(h, 0.8, PITCH, d0) == 0.0)


def _dimple(W=12, H=10, z=6e-3, depth=1.5e-3):
    y, x = np.mgrid[0:H, 0:W]
    r2 = ((x + 0.5) - W / 2) ** 2 + ((y + 0.5) - H / 2) ** 2
    return z - depth * np.exp(-r2 / 8.0)


def test_lights_add_up_and_bounces_only_add_light():
    """Each path ends at one LED at most, so with the same random numbers
    the image under four lit LEDs is the sum of the images with one LED lit
    and the other three dark (still in place, so the paths are the same);
    more bounces only add light (a path that would have ended on the
    membrane may reach an LED later), and a flat membrane reflects once."""
    from paper_2405_02914_gb300 import inputs as I
    h = _dimple()
    H, W = h.shape
    leds = I.sensor_leds(W, H, PITCH, 6e-3)
    alb = I.base_texture(W, H, seed=3).astype(np.float64)
    all4 = RO.render(h, alb, PITCH, RO.make_desc(leds, 32, 4, 0.0, 77))
    parts = sum(RO.render(h, alb, PITCH, RO.make_desc([l if m == k else (l[0], l[1], l[2], (0.0, 0.0, 0.0))
                                                       for m, l in enumerate(leds)], 32, 4, 0.0, 77))
                for k in range(4))
    assert np.abs(all4 - parts).max() < 1e-12
    one = RO.render(h, alb, PITCH, RO.make_desc(leds, 32, 1, 0.0, 77))
    assert np.all(all4 >= one) and (all4 - one).max() > 0
    flat = _flat(W, H, 6e-3)
    assert np.array_equal(RO.render(flat, alb, PITCH, RO.make_desc(leds, 32, 4, 0.0, 5)),
                          RO.render(flat, alb, PITCH, RO.make_desc(leds, 32, 1, 0.0, 5)))


def test_uniforms_are_24_bit_and_uniform():
    u = np.array([RO.uniform(9, k) for k in range(20000)])
    assert np.all(u >= 0) and np.all(u < 1) and np.all(u * 2 ** 24 == np.round(u * 2 ** 24))
    assert abs(u.mean() - 0.5) < 0.01 and abs(u.var() - 1 / 12) < 0.005
    assert RO.uniform(9, 0) != RO.uniform(10, 0)


def test_mse_psnr_closed_forms():
    rng = np.random.default_rng(0)
    a = rng.uniform(0, 1, (20, 17, 3))
    m, p = RO.mse_psnr(a, a + 0.05, 1.0)
    assert m == pytest.approx(0.0025, rel=1e-12) and p == pytest.approx(10 * math.log10(1 / 0.0025), rel=1e-12)
    m, p = RO.mse_psnr(a, a, 1.0)
    assert m == 0.0 and math.isinf(p)


def _gauss_mean(x):
    """Window means by separable convolution with the normalised 11-tap
    Gaussian (sigma 1.5), valid part only."""
    g = np.exp(-((np.arange(11) - 5) ** 2) / (2 * 1.5 ** 2))
    g /= g.sum()
    rows = np.apply_along_axis(lambda r: np.convolve(r, g[::-1], mode="valid"), 1, x)
    return np.apply_along_axis(lambda c: np.convolve(c, g[::-1], mode="valid"), 0, rows)


def test_ssim_closed_forms():
    rng = np.random.default_rng(1)
    a = rng.uniform(0, 1, (24, 20))
    assert RO.ssim(a, a, 1.0) == pytest.approx(1.0, abs=1e-12)
    assert RO.ssim(a, 1 - a, 1.0) == pytest.approx(RO.ssim(1 - a, a, 1.0), abs=1e-14)
    c1 = 0.01 ** 2
    # constant images: only the luminance term is left
    assert RO.ssim(np.full((15, 13), 0.3), np.full((15, 13), 0.6), 1.0) == pytest.approx(
        (2 * 0.3 * 0.6 + c1) / (0.3 ** 2 + 0.6 ** 2 + c1), rel=1e-12)
    # a constant offset keeps variance and covariance: the luminance term of each window
    mu = _gauss_mean(a)
    want = np.mean((2 * mu * (mu + 0.2) + c1) / (mu ** 2 + (mu + 0.2) ** 2 + c1))
    assert RO.ssim(a, a + 0.2, 1.0) == pytest.approx(want, rel=1e-10)
    # channels are averaged
    b = rng.uniform(0, 1, (24, 20))
    both = RO.ssim(np.stack([a, b], -1), np.stack([a + 0.2, b], -1), 1.0)
    assert both == pytest.approx(0.5 * (want + 1.0), rel=1e-10)
