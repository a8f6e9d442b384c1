"""Float64 statement of the learned propagation surrogate (test infrastructure).

The network, its loss, its gradient by plain backpropagation and the Adam
update, written from their definitions with numpy.  ``q`` (optional) is
applied where the CUDA path stores a value in bfloat16 -- the features, the
weights, every hidden activation, the output gradient and each layer's
input gradient -- so that both sides take those roundings at the same
points; with ``q=None`` everything stays float64 (the finite-difference
pin).  Only the test-suite and the benchmark's CPU leg use this module.
"""
from __future__ import annotations

import numpy as np

from . import conv3x3

LAYERS = ((16, 32), (32, 32), (32, 32), (32, 16))
FLOW_SCALE = 4.0


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), via float32."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _id(a):
    return a


def split_params(p):
    """Flat parameter vector -> [(w [9, Cout, Cin], b [Cout]), ...]."""
    out, k = [], 0
    for cin, cout in LAYERS:
        nw = 9 * cout * cin
        out.append((np.asarray(p[k:k + nw], dtype=np.float64).reshape(9, cout, cin),
                    np.asarray(p[k + nw:k + nw + cout], dtype=np.float64)))
        k += nw + cout
    return out


def features(eta, dmu, s0):
    """s0: [n, H, W, 4] (w, rho) -> [n, H, W, 16]: w / (4 dmu), rho, eta_x, eta_y, zeros."""
    s0 = np.asarray(s0, dtype=np.float64)
    n, H, W, _ = s0.shape
    x = np.zeros((n, H, W, 16))
    x[..., 0:3] = s0[..., 0:3] / (FLOW_SCALE * dmu[None, ..., None])
    x[..., 3] = s0[..., 3]
    x[..., 4] = eta[None, ..., 0]
    x[..., 5] = eta[None, ..., 1]
    return x


def conv3x3_dgrad(dy, w):
    """Input gradient of y = conv3x3(x, w): dx[n, i, j, ci] = sum over taps and
    output channels of w[tap, co, ci] dy[n, i - dy + 1, j - dx + 1, co] (the
    output pixels whose window held (i, j)), zero outside."""
    dy = np.asarray(dy, dtype=np.float64)
    N, H, W, Cout = dy.shape
    Cin = w.shape[2]
    dyp = np.zeros((N, H + 2, W + 2, Cout))
    dyp[:, 1:H + 1, 1:W + 1] = dy
    dx = np.zeros((N, H, W, Cin))
    for a in range(3):
        for b in range(3):
            dx += dyp[:, 2 - a:2 - a + H, 2 - b:2 - b + W, :] @ w[3 * a + b]
    return dx


def conv3x3_wgrad(x, dy):
    """Weight and bias gradients: dw[tap, co, ci] = sum_p dy[p, co] x[p + off(tap), ci]."""
    x = np.asarray(x, dtype=np.float64); dy = np.asarray(dy, dtype=np.float64)
    N, H, W, Cin = x.shape
    Cout = dy.shape[3]
    xp = np.zeros((N, H + 2, W + 2, Cin))
    xp[:, 1:H + 1, 1:W + 1] = x
    dw = np.zeros((9, Cout, Cin))
    for a in range(3):
        for b in range(3):
            dw[3 * a + b] = np.einsum("nhwo,nhwi->oi", dy, xp[:, a:a + H, b:b + W, :])
    return dw, dy.sum(axis=(0, 1, 2))


def forward(x0, params, q=None):
    """Activations [x0, a1, a2, a3] and the float output of the 4 layers."""
    q = q or _id
    acts = [q(x0)]
    layers = split_params(params)
    for l, (w, b) in enumerate(layers):
        y = conv3x3(acts[-1], q(w), b, relu=l < 3)
        if l < 3:
            acts.append(q(y))
        else:
            return acts, y


def residual_target(eta, dmu, s0, target):
    """The target prediction in the network's units (channels 0..3)."""
    t = np.zeros(np.asarray(s0).shape[:3] + (16,))
    t[..., 0:3] = (np.asarray(target)[..., 0:3] - np.asarray(s0)[..., 0:3]) / (FLOW_SCALE * dmu[None, ..., None])
    t[..., 3] = np.asarray(target)[..., 3] - np.asarray(s0)[..., 3]
    return t


def loss_and_grads(x0, params, t, q=None):
    """Mean squared error over the 4 used output channels, and its gradient
    with respect to the flat parameter vector (backpropagation)."""
    qq = q or _id
    acts, y = forward(x0, params, q)
    n_px = y.shape[0] * y.shape[1] * y.shape[2]
    e = (y - t)[..., :4]
    loss = float((e ** 2).sum() / (4 * n_px))
    dy = np.zeros_like(y)
    dy[..., :4] = 2.0 * e / (4 * n_px)
    dy = qq(dy)
    layers = split_params(params)
    grads = [None] * 4
    for l in range(3, -1, -1):
        w, _ = layers[l]
        gw, gb = conv3x3_wgrad(acts[l], dy)
        grads[l] = (gw, gb)
        if l == 0:
            break
        dx = qq(conv3x3_dgrad(dy, qq(w)))
        dy = np.where(acts[l] > 0, dx, 0.0)
    return loss, np.concatenate([np.concatenate([g[0].ravel(), g[1]]) for g in grads])


def adam(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (t counts from 1); returns new (p, m, v)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
