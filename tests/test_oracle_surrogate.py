"""Pins of the oracle's surrogate network pieces: the backward convolutions
are the adjoints of the forward one, the loss gradient matches central
finite differences, Adam under a constant gradient steps by lr sign(g), and
the bfloat16 rounding is the IEEE-style round-to-nearest-even."""
import numpy as np

from oracle import conv3x3
from oracle import surrogate as S


def test_backward_convolutions_are_adjoints():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 5, 7, 3)); w = rng.normal(size=(9, 4, 3)); dy = rng.normal(size=(2, 5, 7, 4))
    lhs = float((conv3x3(x, w) * dy).sum())
    gw, gb = S.conv3x3_wgrad(x, dy)
    assert abs(lhs - float((w * gw).sum())) < 1e-9 * max(1.0, abs(lhs))
    assert abs(lhs - float((x * S.conv3x3_dgrad(dy, w)).sum())) < 1e-9 * max(1.0, abs(lhs))
    np.testing.assert_allclose(gb, dy.sum(axis=(0, 1, 2)))


def test_loss_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    n_params = sum(9 * ci * co + co for ci, co in S.LAYERS)
    p = rng.normal(size=n_params) * 0.15
    x0 = rng.normal(size=(1, 4, 5, 16)); x0[..., 6:] = 0.0
    t = rng.normal(size=(1, 4, 5, 16)) * 0.1
    loss, g = S.loss_and_grads(x0, p, t)
    idx = rng.choice(n_params, size=40, replace=False)
    h = 1e-6
    for k in idx:
        pp = p.copy(); pp[k] += h
        pm = p.copy(); pm[k] -= h
        fd = (S.loss_and_grads(x0, pp, t)[0] - S.loss_and_grads(x0, pm, t)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g).max()), (k, fd, g[k])


def test_adam_under_constant_gradient():
    g = np.array([0.3, -2.0, 1e-3])
    p = np.zeros(3); m = np.zeros(3); v = np.zeros(3)
    for t in range(1, 6):
        p_new, m, v = S.adam(p, g, m, v, t, lr=0.01)
        # bias-corrected moments equal g and g^2 exactly: the step is lr g / (|g| + eps)
        np.testing.assert_allclose(p_new - p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-9)
        p = p_new


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 3.0e-40, 65504.0], dtype=np.float32)
    out = S.bf16(vals)
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties go to the even mantissa (1)
    assert out[0] == 1.0 and out[1] == 1.0 and out[2] == 1.0 + 2 ** -6 and out[3] == -2.5
    assert out[5] == 65536.0
    # every result has a zero low half
    assert (np.asarray(out, dtype=np.float32).view(np.uint32) & 0xFFFF == 0).all()
