"""Pins of the FP64 surrogate oracle against things other than itself:
scipy's 2-D correlation, torch's CPU conv2d / nearest upsampling / autograd
in FP64 (an independent construction of the whole network), central finite
differences, hand-worked loss values, torch's BF16 rounding and Adam."""
import numpy as np
import pytest
from scipy import signal

from oracle import surrogate_oracle as so
from paper_2405_02914_gb300 import inputs

torch = pytest.importorskip("torch")


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


@pytest.mark.parametrize("stride", [1, 2])
def test_conv_matches_scipy_correlate(stride):
    B, H, W, C, O = 2, 8, 6, 3, 4
    x = _rand((B, H, W, C), 1)
    Wt = _rand((O, 3, 3, C), 2)          # asymmetric taps: a ky/kx swap fails
    b = _rand(O, 3)
    out = so.conv3x3(x, Wt, b, stride)
    ref = np.zeros((B, H, W, O))
    for bb in range(B):
        for o in range(O):
            ref[bb, :, :, o] = b[o] + sum(signal.correlate2d(x[bb, :, :, c], Wt[o, :, :, c], mode="same",
                                                             boundary="fill") for c in range(C))
    ref = ref[:, ::stride, ::stride, :]
    assert out.shape == ref.shape
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-12)


def test_conv_delta_and_shift_kernels():
    x = _rand((1, 6, 6, 2), 4)
    Wt = np.zeros((2, 3, 3, 2))
    Wt[0, 1, 1, 0] = 1.0                 # identity on channel 0
    Wt[1, 0, 2, 1] = 1.0                 # out(y, x) = in(y-1, x+1) on channel 1
    out = so.conv3x3(x, Wt, np.zeros(2), 1)
    np.testing.assert_array_equal(out[..., 0], x[..., 0])
    np.testing.assert_array_equal(out[0, 1:, :-1, 1], x[0, :-1, 1:, 1])
    assert np.all(out[0, 0, :, 1] == 0) and np.all(out[0, :, -1, 1] == 0)


def test_upsample_gradient_is_adjoint():
    a = _rand((2, 3, 4, 5), 5)
    d = _rand((2, 6, 8, 5), 6)
    assert abs((so.up2(a) * d).sum() - (a * so.up2_grad(d)).sum()) < 1e-10
    np.testing.assert_array_equal(so.up2(a)[:, 1::2, ::2], a)


def test_loss_hand_worked():
    y = np.array([[[[1.0, 2.0, 2.0, 0.0], [0.0, 0.0, 0.0, 5.0]]]])
    t = np.zeros((1, 1, 2, 3))
    # pixel 0: |r|^2 = 9, e = 3, (0 - 3)^2 = 9 -> 18; pixel 1 masked out
    L, g = so.loss_and_grad_y(y, t, np.array([[[1.0, 0.0]]]))
    assert L == pytest.approx(18.0, abs=1e-14)
    np.testing.assert_allclose(g[0, 0, 0], [2.0, 4.0, 4.0, -6.0])
    np.testing.assert_array_equal(g[0, 0, 1], 0.0)
    # both pixels: (18 + 25) / 2
    L2, _ = so.loss_and_grad_y(y, t, np.ones((1, 1, 2)))
    assert L2 == pytest.approx(21.5, abs=1e-14)


def _torch_net(p, x):
    """The network of include/tsurr.h built from torch CPU ops (NCHW, FP64)."""
    import torch.nn.functional as F
    params = []
    off = 0
    for cin, cout in inputs.SURR_CONVS:
        nw = cout * 9 * cin
        w = p[off:off + nw].view(cout, 3, 3, cin).permute(0, 3, 1, 2)
        params.append((w, p[off + nw:off + nw + cout]))
        off += nw + cout
    h = torch.zeros(x.shape[0], 16, x.shape[1], x.shape[2], dtype=torch.float64)
    h[:, :12] = x.permute(0, 3, 1, 2)
    a0 = F.relu(F.conv2d(h, *params[0], padding=1))
    a1 = F.relu(F.conv2d(a0, *params[1], stride=2, padding=1))
    a2 = F.relu(F.conv2d(a1, *params[2], stride=2, padding=1))
    a3 = F.relu(F.conv2d(a2, *params[3], stride=2, padding=1))
    a4 = F.relu(F.conv2d(a3, *params[4], padding=1))
    up = lambda a: F.interpolate(a, scale_factor=2, mode="nearest")  # noqa: E731
    a5 = F.relu(F.conv2d(up(a4), *params[5], padding=1) + a2)
    a6 = F.relu(F.conv2d(up(a5), *params[6], padding=1) + a1)
    a7 = F.relu(F.conv2d(up(a6), *params[7], padding=1) + a0)
    y = F.conv2d(a7, *params[8], padding=1)
    return y[:, :4].permute(0, 2, 3, 1)


def _torch_loss(y, t, m):
    r = y[..., :3] - t
    e = torch.sqrt((r * r).sum(-1)).detach()
    return (m * ((r * r).sum(-1) + (y[..., 3] - e) ** 2)).sum() / m.sum()


def _case(B=2, H=16, W=8, seed=0):
    p = inputs.surrogate_params(seed, bias_std=0.1, scale_last=1.0).astype(np.float64)
    x, t, m = inputs.surrogate_batch(seed, B, H, W)
    return p, x.astype(np.float64), t.astype(np.float64), m.astype(np.float64)


def test_forward_matches_torch():
    p, x, _, _ = _case()
    y, _ = so.forward(p, x)
    yt = _torch_net(torch.from_numpy(p), torch.from_numpy(x)).numpy()
    assert np.abs(yt).max() > 0.1
    np.testing.assert_allclose(y, yt, rtol=1e-10, atol=1e-11)


def test_backward_matches_torch_autograd():
    p, x, t, m = _case(seed=1)
    L, g = so.backward(p, x, t, m)
    pt = torch.from_numpy(p).requires_grad_(True)
    Lt = _torch_loss(_torch_net(pt, torch.from_numpy(x)), torch.from_numpy(t), torch.from_numpy(m))
    Lt.backward()
    gt = pt.grad.numpy()
    assert L == pytest.approx(Lt.item(), rel=1e-12)
    assert np.abs(gt).max() > 1e-3
    np.testing.assert_allclose(g, gt, rtol=1e-8, atol=1e-12 * np.abs(gt).max())


def test_backward_central_differences():
    p, x, t, m = _case(B=1, H=8, W=8, seed=2)
    L0, g = so.backward(p, x, t, m)
    rng = np.random.default_rng(3)
    y0, _ = so.forward(p, x)
    e0 = np.sqrt(((y0[..., :3] - t) ** 2).sum(-1))      # the indicator target is held constant

    def loss_at(q):
        y, _ = so.forward(q, x)
        return (m * (((y[..., :3] - t) ** 2).sum(-1) + (y[..., 3] - e0) ** 2)).sum() / m.sum()

    assert loss_at(p) == pytest.approx(L0, rel=1e-13)

    # directional derivative along a random direction
    d = rng.standard_normal(p.size)
    h = 1e-6
    fd = (loss_at(p + h * d) - loss_at(p - h * d)) / (2 * h)
    assert fd == pytest.approx(g @ d, rel=1e-6)
    # single coordinates in every layer (the largest-gradient weight of each)
    off = 0
    for cin, cout in inputs.SURR_CONVS:
        nw = cout * 9 * cin
        k = off + int(np.argmax(np.abs(g[off:off + nw])))
        e = np.zeros(p.size)
        e[k] = 1.0
        fdk = (loss_at(p + 1e-5 * e) - loss_at(p - 1e-5 * e)) / 2e-5
        assert fdk == pytest.approx(g[k], rel=1e-5, abs=1e-9)
        off += nw + cout


def test_round_bf16_matches_torch():
    v = np.concatenate([_rand(4000, 7) * 10.0 ** np.random.default_rng(8).integers(-6, 6, 4000),
                        [1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -1.0 - 2.0 ** -8, 0.0, -0.0]])
    ours = so.round_bf16(v)
    ref = torch.from_numpy(v.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(ours, ref)
    assert ours[-5] == 1.0 and ours[-4] == 1.0 + 2.0 ** -6


def test_adam_matches_torch():
    p0 = _rand(50, 9)
    grads = [_rand(50, 10 + i) for i in range(4)]
    pt = torch.tensor(p0, requires_grad=True)
    opt = torch.optim.Adam([pt], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    p, m1, m2 = p0.copy(), np.zeros(50), np.zeros(50)
    for i, gi in enumerate(grads):
        pt.grad = torch.from_numpy(gi)
        opt.step()
        p, m1, m2 = so.adam(p, gi, m1, m2, i + 1, 1e-2)
    np.testing.assert_allclose(p, pt.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_bf16_mode_only_rounds():
    p, x, t, m = _case(seed=4)
    y64, _ = so.forward(p, x)
    y16, _ = so.forward(p, x, bf16=True)
    rel = np.linalg.norm(y16 - y64) / np.linalg.norm(y64)
    assert 1e-5 < rel < 3e-2
    L64, g64 = so.backward(p, x, t, m)
    L16, g16 = so.backward(p, x, t, m, bf16=True)
    cos = g16 @ g64 / np.linalg.norm(g16) / np.linalg.norm(g64)
    assert cos > 0.999
