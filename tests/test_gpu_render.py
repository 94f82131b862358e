"""The sensor-image path tracer and image metrics on the GPU against the FP64
oracle (oracle/render_oracle.c).  Both draw the same SplitMix64 uniforms for
every sample, so a GPU path and an oracle path coincide unless an FP32
rounding flips one of its geometric decisions (which LED, floor or membrane
is met first, a bisection step); a flipped sample moves its pixel by at most
throughput x radiance / spp.  The tolerance: pixel values within 1e-4
except a few per cent of them, each within 3 / spp, and the mean difference
below 1e-3."""
import numpy as np
import pytest
import torch

from oracle import render_oracle as RO
from paper_2405_02914_gb300 import inputs as I
from paper_2405_02914_gb300 import tsim as T

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _dimple(W, H, pitch, z, depth, rad):
    y, x = np.mgrid[0:H, 0:W]
    r2 = (((x + 0.5) - W / 2) ** 2 + ((y + 0.5) - H / 2) ** 2) * pitch ** 2
    return (z - depth * np.exp(-r2 / (2 * rad ** 2))).astype(np.float32)


def _gpu(h, alb, pitch, leds, spp, bounces, seed):
    d = T.render_desc(leds, spp, bounces, 0.0, seed)
    out = T.tsim_render(torch.from_numpy(h).to(DEV), torch.from_numpy(alb).to(DEV), pitch, d)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def _oracle(h, alb, pitch, leds, spp, bounces, seed):
    return RO.render(h.astype(np.float64), alb.astype(np.float64), pitch, RO.make_desc(leds, spp, bounces, 0.0, seed))


def _agree(g, o, spp):
    d = np.abs(g - o)
    assert d.mean() < 1e-3, d.mean()
    assert np.mean(d > 1e-4) < 0.03, np.mean(d > 1e-4)
    assert d.max() <= 3.0 / spp, d.max()


@pytest.mark.parametrize("colors,bounces", [("gelsight", 4), ("white", 1)])
def test_render_matches_oracle(colors, bounces):
    W, H, pitch = 24, 20, 0.3e-3
    h = _dimple(W, H, pitch, 3e-3, 0.6e-3, 1.2e-3)
    alb = I.base_texture(W, H, seed=2)
    leds = I.sensor_leds(W, H, pitch, 3e-3, colors)
    spp = 64
    g = _gpu(h, alb, pitch, leds, spp, bounces, 11)
    o = _oracle(h, alb, pitch, leds, spp, bounces, 11)
    assert o.max() > 0.05                       # lit
    _agree(g, o, spp)


def test_render_of_a_simulated_surface_matches_oracle():
    """The membrane of an IMPM press (the readout of tsim_read_surface)."""
    sc = I.scene_small(cx=16, cy=16, cz=4, n_press=60, press=0.5e-3, mu=0.6)
    sim = T.Sim(sc)
    sim.step(60)
    h, _ = sim.surface()
    sim.close()
    h = np.ascontiguousarray(h, dtype=np.float32)
    Hh, Ww = h.shape
    pitch = sc.readout_pitch
    alb = I.base_texture(Ww, Hh, seed=4)
    leds = I.sensor_leds(Ww, Hh, pitch, sc.gel.height, "gelsight")
    assert h.min() < sc.gel.height - 0.2e-3            # pressed
    g = _gpu(h, alb, pitch, leds, 32, 4, 3)
    o = _oracle(h, alb, pitch, leds, 32, 4, 3)
    _agree(g, o, 32)


def test_full_size_render_properties():
    """128 x 128 pixels at 128 samples (the paper's sample count): the whole
    image against the oracle; LEDs add up (one lit, three dark in place, same
    random numbers), extra bounces only add light, a flat membrane reflects
    once."""
    W = H = 128
    pitch = 0.3125e-3
    h = _dimple(W, H, pitch, 10e-3, 1e-3, 3e-3)
    alb = I.base_texture(W, H, seed=5)
    leds = I.sensor_leds(W, H, pitch, 10e-3, "gelsight")
    full = _gpu(h, alb, pitch, leds, 128, 4, 21)
    _agree(full, _oracle(h, alb, pitch, leds, 128, 4, 21), 128)
    parts = sum(_gpu(h, alb, pitch, [l if m == k else (l[0], l[1], l[2], (0.0, 0.0, 0.0))
                                     for m, l in enumerate(leds)], 128, 4, 21) for k in range(4))
    assert np.abs(full - parts).max() < 1e-5
    one = _gpu(h, alb, pitch, leds, 128, 1, 21)
    assert np.all(full >= one - 1e-6) and (full - one).max() > 0
    flat = np.full((H, W), 10e-3, dtype=np.float32)
    assert np.array_equal(_gpu(flat, alb, pitch, leds, 128, 4, 9), _gpu(flat, alb, pitch, leds, 128, 1, 9))


def test_image_metrics_match_oracle():
    rng = np.random.default_rng(7)
    a = rng.uniform(0, 1, (40, 36, 3)).astype(np.float32)
    b = np.clip(a + rng.normal(0, 0.05, a.shape), 0, 1).astype(np.float32)
    ta, tb = torch.from_numpy(a).to(DEV), torch.from_numpy(b).to(DEV)
    mse, psnr, ssim = T.tsim_image_metrics(ta, tb, 1.0)
    om, op = RO.mse_psnr(a, b, 1.0)
    assert mse == pytest.approx(om, rel=1e-9) and psnr == pytest.approx(op, rel=1e-9)
    assert ssim == pytest.approx(RO.ssim(a, b, 1.0), rel=1e-5)
    mse, psnr, ssim = T.tsim_image_metrics(ta, ta, 1.0)
    assert mse == 0.0 and np.isinf(psnr) and ssim == pytest.approx(1.0, abs=1e-6)


def test_render_rejects_host_arrays_and_bad_descriptors():
    h = torch.zeros((8, 8), device=DEV)
    alb = torch.zeros((8, 8, 3), device=DEV)
    d = T.render_desc(I.sensor_leds(8, 8, 1e-3, 2e-3), 4, 2)
    with pytest.raises(T.TsimError):
        T.tsim_render(h.cpu(), alb, 1e-3, d)
    bad = T.render_desc(I.sensor_leds(8, 8, 1e-3, 2e-3), 4, 0)
    with pytest.raises(T.TsimError):
        T.tsim_render(h, alb, 1e-3, bad)
