"""Surrogate kernels (libtsim.so, include/tsurr.h) against the FP64 oracle.

Tolerances come from the arithmetic: the kernels store activations, weights
and pre-activation gradients in BF16 (relative rounding 2^-9) and accumulate
in FP32.  Against the oracle run with BF16 rounding at the same points the
remaining differences are FP32 accumulation order plus the odd BF16 value
that rounds the other way (relative L2 <= 5e-3 on outputs, 1e-2 on
gradients).  Against the plain FP64 oracle the nine layers of BF16 rounding
allow 3e-2 on outputs and a gradient cosine >= 0.995 per layer (BF16
rounding alone gives 0.9986 on the 2x2-pixel deep layers of the smallest
cases, measured with the oracle's BF16 mode).
"""
import numpy as np
import pytest

from oracle import surrogate_oracle as so
from paper_2405_02914_gb300 import inputs as I
from paper_2405_02914_gb300 import tsurr as S

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def _net(B, H, W, p):
    net = S.tsurr_create(B, H, W)
    S.tsurr_set_params(net, p)
    return net


def _layer_slices():
    out, off = [], 0
    for cin, cout in I.SURR_CONVS:
        nw = cout * 9 * cin
        out.append((slice(off, off + nw), slice(off + nw, off + nw + cout), (cout, 3, 3, cin)))
        off += nw + cout
    return out


@pytest.mark.parametrize("B,H,W", [(1, 8, 8), (3, 16, 24), (2, 32, 32)])
def test_forward_matches_oracle(B, H, W):
    p = I.surrogate_params(11, bias_std=0.1, scale_last=1.0)
    x, _, _ = I.surrogate_batch(12, B, H, W)
    net = _net(B, H, W, p)
    try:
        y = S.tsurr_forward(net, x)
    finally:
        S.tsurr_destroy(net)
    y16, _ = so.forward(p, x, bf16=True)
    y64, _ = so.forward(p, x)
    assert y.shape == (B, H, W, 4) and np.all(np.isfinite(y))
    assert _rel(y, y16) <= 5e-3
    assert _rel(y, y64) <= 3e-2
    assert np.abs(y - y16).max() <= 3e-2 * np.abs(y16).max()


# (2, 16, 16), (3, 16, 24), (1, 32, 8): weight gradients of the narrow layers
# on mma.sync; (2, 32, 48): layers 0, 7, 8 on tcgen05 with three 16-pixel
# row segments per output row; (1, 128, 128): every layer on tcgen05
@pytest.mark.parametrize("B,H,W", [(2, 16, 16), (3, 16, 24), (1, 32, 8), (2, 32, 48), (1, 128, 128)])
def test_backward_matches_oracle(B, H, W):
    p = I.surrogate_params(21, bias_std=0.1, scale_last=1.0)
    x, t, m = I.surrogate_batch(22, B, H, W)
    net = _net(B, H, W, p)
    try:
        L = S.tsurr_backward(net, x, t, m)
        g = S.tsurr_get_grads(net)
    finally:
        S.tsurr_destroy(net)
    L16, g16 = so.backward(p, x, t, m, bf16=True)
    L64, g64 = so.backward(p, x, t, m)
    assert L == pytest.approx(L16, rel=5e-3)
    assert L == pytest.approx(L64, rel=3e-2)
    for li, (ws, bs, shape) in enumerate(_layer_slices()):
        assert _rel(g[ws], g16[ws]) <= 1e-2, li
        assert _rel(g[bs], g16[bs]) <= 1e-2, li
        cos = g[ws] @ g64[ws] / np.linalg.norm(g[ws]) / np.linalg.norm(g64[ws])
        assert cos >= 0.995, (li, cos)
    # padded input channels and unused output rows get exactly zero gradient
    ws0, _, shape0 = _layer_slices()[0]
    assert np.all(g[ws0].reshape(shape0)[..., 12:] == 0)
    ws8, bs8, shape8 = _layer_slices()[-1]
    assert np.all(g[ws8].reshape(shape8)[4:] == 0) and np.all(g[bs8][4:] == 0)


def test_adam_step_matches_oracle():
    B, H, W = 2, 16, 16
    p = I.surrogate_params(31, bias_std=0.1, scale_last=1.0)
    x, t, m = I.surrogate_batch(32, B, H, W)
    lr = 1e-3
    net = _net(B, H, W, p)
    try:
        S.tsurr_backward(net, x, t, m)
        S.tsurr_adam(net, lr, 0.9, 0.999, 1e-8, 1)
        p1 = S.tsurr_get_params(net)
    finally:
        S.tsurr_destroy(net)
    _, g16 = so.backward(p, x, t, m, bf16=True)
    q, _, _ = so.adam(p.astype(np.float64), g16, 0.0, 0.0, 1, lr)
    # at t = 1 the step is lr * g / (|g| + eps): the oracle fixes it wherever the
    # gradient is well above the BF16 noise of the kernels' gradient
    big = np.abs(g16) > 0.1 * np.sqrt(np.mean(g16 ** 2))
    assert big.sum() > 1000
    np.testing.assert_allclose((p1 - p)[big], (q - p)[big], atol=2e-3 * lr, rtol=0)
    assert np.all(np.abs(p1 - p) <= lr + 1e-7)


def test_training_reduces_loss():
    B, H, W = 4, 32, 32
    p = I.surrogate_params(41)
    x, t, m = I.surrogate_batch(42, B, H, W)
    t = (0.3 * x[..., :1] * np.array([1.0, -0.5, 2.0], np.float32)).astype(np.float32)   # learnable map
    net = _net(B, H, W, p)
    try:
        losses = []
        for step in range(1, 81):
            losses.append(S.tsurr_backward(net, x, t, m))
            S.tsurr_adam(net, 1e-3, 0.9, 0.999, 1e-8, step)
    finally:
        S.tsurr_destroy(net)
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.2 * losses[0], (losses[0], losses[-1])


def test_full_size_batch_invariance_and_sampled_oracle():
    """Inference batch 256 at 128x128: each sample's output is bit-identical to
    a batch-1 run (no cross-sample terms, same accumulation order), and one
    sampled image matches the oracle."""
    B, H, W = 256, 128, 128
    p = I.surrogate_params(51, bias_std=0.05)
    x, _, _ = I.surrogate_batch(52, B, H, W)
    net = S.tsurr_create(B, H, W)
    try:
        S.tsurr_set_params(net, p)
        y = S.tsurr_forward(net, x)
        for b in (0, 97, 255):
            yb = S.tsurr_forward(net, np.ascontiguousarray(x[b:b + 1]))
            np.testing.assert_array_equal(yb[0], y[b])
    finally:
        S.tsurr_destroy(net)
    y16, _ = so.forward(p, x[97:98], bf16=True)
    assert _rel(y[97:98], y16) <= 5e-3


def test_device_pointers_and_bad_batch():
    torch = pytest.importorskip("torch")
    B, H, W = 2, 16, 16
    p = I.surrogate_params(61, bias_std=0.1)
    x, t, m = I.surrogate_batch(62, B, H, W)
    net = _net(B, H, W, p)
    try:
        yh = S.tsurr_forward(net, x)
        xd = torch.from_numpy(x).cuda()
        yd = torch.empty((B, H, W, 4), dtype=torch.float32, device="cuda")
        S.tsurr_forward(net, xd, out=yd)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(yd.cpu().numpy(), yh)
        Lh = S.tsurr_backward(net, x, t, m)
        Ld = S.tsurr_backward(net, xd, torch.from_numpy(t).cuda(), torch.from_numpy(m).cuda())
        assert Ld == pytest.approx(Lh, rel=1e-6)     # FP64 sum of FP32 partials, any order
        with pytest.raises(S._t.TsimError):
            S.tsurr_forward(net, np.zeros((3, H, W, 12), np.float32))
    finally:
        S.tsurr_destroy(net)


def test_serving_helpers_match_their_definitions():
    """The feature assembly and the indicator reduction of the serving path
    (tsurr_features, tsurr_indicator) against their definitions written out
    in numpy on random inputs of a ragged size."""
    import torch
    rng = np.random.default_rng(3)
    B, H, W = 5, 24, 40
    h = rng.standard_normal((B, H, W)).astype(np.float32)
    sc = rng.standard_normal((B, 9)).astype(np.float32)
    x = S.tsurr_features(torch.from_numpy(h).cuda(), torch.from_numpy(sc).cuda()).cpu().numpy()
    px = ((np.arange(W, dtype=np.float32) + np.float32(0.5)) / np.float32(W)) * np.float32(2) - np.float32(1)
    py = ((np.arange(H, dtype=np.float32) + np.float32(0.5)) / np.float32(H)) * np.float32(2) - np.float32(1)
    ref = np.empty((B, H, W, 12), np.float32)
    ref[..., 0] = h
    ref[..., 1] = px[None, None, :]
    ref[..., 2] = py[None, :, None]
    ref[..., 3:] = sc[:, None, None, :]
    assert np.array_equal(x, ref)
    y = rng.standard_normal((B, H, W, 4)).astype(np.float32)
    press = rng.uniform(0.3, 1.0, B).astype(np.float32)
    ind = S.tsurr_indicator(torch.from_numpy(y).cuda(), torch.from_numpy(press).cuda()).cpu().numpy()
    want = np.sqrt((y[..., 3].astype(np.float64) ** 2).mean(axis=(1, 2))) / press
    assert np.allclose(ind, want, rtol=1e-5)
