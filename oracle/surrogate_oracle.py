"""FP64 CPU oracle of the learned surface surrogate (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py may import this module; it
shares no code with the CUDA path.  The network is not part of the paper's
method (a project addition); its definition is the architecture and loss
stated in include/tsurr.h, restated here from that description:

  * every layer is a 3x3 convolution with zero padding 1 on NHWC images,
    out[b,y,x,o] = bias[o] + sum_{ky,kx,c} W[o,ky,kx,c] in[b, s*y+ky-1, s*x+kx-1, c];
  * layers 5..7 read the nearest x2 upsampling of their input and add the
    encoder activation of the same size (a2, a1, a0) before the ReLU;
  * the input has 12 channels zero-padded to 16, the last layer has 16
    output rows of which the first 4 are the network output;
  * loss = sum_p m_p (|y_p[0:3]-t_p|^2 + (y_p[3]-e_p)^2) / sum_p m_p with
    e_p = |y_p[0:3]-t_p| held constant.

Parity pins (tests/test_surrogate_pins.py): the convolution against scipy's
correlate, the whole forward and its gradient against torch's CPU conv2d and
autograd in FP64, central finite differences, and the loss on a hand-worked
case.  ``bf16=True`` rounds at the points where the GPU kernels store BF16
(inputs, weights, stored activations, pre-activation gradients) so that the
GPU can be compared at a tighter tolerance; the FP64 arithmetic is otherwise
unchanged.
"""
from __future__ import annotations

import numpy as np

CIN, COUT = 12, 4
# (cin, cout, stride, upsample, relu, skip) -- skip = index of the encoder
# layer whose output is added before the ReLU, or None
ARCH = [
    (16, 32, 1, False, True, None),
    (32, 64, 2, False, True, None),
    (64, 128, 2, False, True, None),
    (128, 256, 2, False, True, None),
    (256, 256, 1, False, True, None),
    (256, 128, 1, True, True, 2),
    (128, 64, 1, True, True, 1),
    (64, 32, 1, True, True, 0),
    (32, 16, 1, False, False, None),
]


def round_bf16(a):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def unflatten(p):
    """Flat FP32/FP64 parameter vector -> [(W[cout,3,3,cin], b[cout])]."""
    p = np.asarray(p, dtype=np.float64)
    out, off = [], 0
    for cin, cout, *_ in ARCH:
        nw = cout * 9 * cin
        out.append((p[off:off + nw].reshape(cout, 3, 3, cin), p[off + nw:off + nw + cout]))
        off += nw + cout
    if off != p.size:
        raise ValueError("parameter vector has %d entries, the network %d" % (p.size, off))
    return out


def flatten(params):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in params])


def conv3x3(x, W, b, stride):
    """Definition above: zero padding 1, output size = input size / stride."""
    B, H, Wd, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    Ho, Wo = H // stride, Wd // stride
    out = np.broadcast_to(b, (B, Ho, Wo, W.shape[0])).copy()
    for ky in range(3):
        for kx in range(3):
            tap = xp[:, ky:ky + stride * Ho:stride, kx:kx + stride * Wo:stride, :]
            out += np.tensordot(tap, W[:, ky, kx, :], axes=([3], [1]))
    return out


def conv3x3_grads(x, W, stride, dout):
    """(dx, dW, db) of conv3x3 for the output gradient dout."""
    B, H, Wd, C = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    Ho, Wo = H // stride, Wd // stride
    dxp = np.zeros_like(xp)
    dW = np.zeros_like(W)
    for ky in range(3):
        for kx in range(3):
            sl = (slice(None), slice(ky, ky + stride * Ho, stride), slice(kx, kx + stride * Wo, stride), slice(None))
            dW[:, ky, kx, :] = np.tensordot(dout, xp[sl], axes=([0, 1, 2], [0, 1, 2]))
            dxp[sl] += np.tensordot(dout, W[:, ky, kx, :], axes=([3], [0]))
    return dxp[:, 1:-1, 1:-1, :], dW, dout.sum(axis=(0, 1, 2))


def up2(x):
    return x.repeat(2, axis=1).repeat(2, axis=2)


def up2_grad(d):
    B, H, W, C = d.shape
    return d.reshape(B, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def _q(a, on):
    return round_bf16(a) if on else a


def forward(p, x, bf16=False):
    """x[B,H,W,12] -> (y[B,H,W,4], cache)."""
    params = unflatten(p)
    x = np.asarray(x, dtype=np.float64)
    B, H, W, _ = x.shape
    h = np.zeros((B, H, W, ARCH[0][0]))
    h[..., :CIN] = x
    h = _q(h, bf16)
    acts = [h]                        # acts[i] = input of layer i; acts[i+1] its output
    pre = []
    for li, ((cin, cout, stride, up, relu, skip), (Wl, bl)) in enumerate(zip(ARCH, params)):
        inp = up2(acts[li]) if up else acts[li]
        z = conv3x3(inp, _q(Wl, bf16), bl, stride)
        if skip is not None:
            z = z + acts[skip + 1]
        pre.append(z)
        a = np.maximum(z, 0.0) if relu else z
        acts.append(_q(a, bf16) if li < len(ARCH) - 1 else a)
    y = acts[-1][..., :COUT]
    return y, (params, acts, pre, bf16)


def loss_and_grad_y(y, t, m):
    """Loss and dL/dy (the indicator target e held constant)."""
    y = np.asarray(y, np.float64)
    t = np.asarray(t, np.float64)
    m = np.asarray(m, np.float64)
    S = m.sum()
    r = y[..., :3] - t
    e = np.sqrt((r * r).sum(-1))
    ri = y[..., 3] - e
    inv = 1.0 / S if S > 0 else 0.0
    L = (m * ((r * r).sum(-1) + ri * ri)).sum() * inv
    g = np.zeros_like(y)
    g[..., :3] = 2.0 * m[..., None] * r * inv
    g[..., 3] = 2.0 * m * ri * inv
    return L, g


def backward(p, x, t, m, bf16=False):
    """(loss, flat gradient) of the loss above, by reverse-mode differentiation."""
    y, (params, acts, pre, q) = forward(p, x, bf16)
    L, gy = loss_and_grad_y(y, t, m)
    grads = [None] * len(ARCH)
    dacts = [np.zeros_like(a) for a in acts]
    last = acts[-1]
    dlast = np.zeros_like(last)
    dlast[..., :COUT] = gy
    dacts[-1] = dlast
    for li in range(len(ARCH) - 1, -1, -1):
        cin, cout, stride, up, relu, skip = ARCH[li]
        Wl, _ = params[li]
        d = dacts[li + 1]
        if relu:
            d = np.where(pre[li] > 0, d, 0.0)
        d = _q(d, q)
        if skip is not None:
            dacts[skip + 1] = dacts[skip + 1] + d
        inp = up2(acts[li]) if up else acts[li]
        dinp, dW, db = conv3x3_grads(inp, _q(Wl, q), stride, d)
        grads[li] = (dW, db)
        if li > 0:
            dacts[li] = dacts[li] + (up2_grad(dinp) if up else dinp)
    return L, flatten(grads)


def adam(p, g, m1, m2, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One bias-corrected Adam step (Kingma and Ba, Algorithm 1); returns new (p, m1, m2)."""
    m1 = b1 * m1 + (1 - b1) * g
    m2 = b2 * m2 + (1 - b2) * g * g
    mh = m1 / (1 - b1 ** t)
    vh = m2 / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m1, m2
