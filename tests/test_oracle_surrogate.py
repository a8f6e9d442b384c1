"""Pins of the oracle's surrogate network pieces: the backward convolutions
are the adjoints of the forward one, the loss gradient matches central
finite differences, Adam under a constant gradient steps by lr sign(g), the
bfloat16 rounding is the IEEE-style round-to-nearest-even, the features and
the training target match hand-computed values, and the element-wise
gradient tolerance the GPU parity test uses covers a float32 restatement of
the network while rejecting plausible indexing mistakes."""
import numpy as np

from oracle import conv3x3
from oracle import surrogate as S
from tests import surrogate_bounds as SB


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


def test_features_and_target_by_hand():
    # one frame of 1 x 2 pixels with chosen geometry: the features are
    # w / (4 dmu), rho, eta_x, eta_y and ten zeros; the target is the change
    # of the state in the same units
    eta = np.array([[[0.6, 0.0, 0.8], [0.0, -0.28, 0.96]]])
    dmu = np.array([[0.01, 0.02]])
    s0 = np.array([[[[0.04, -0.02, 0.008, 0.5], [0.0, 0.16, -0.08, 0.25]]]])
    x = S.features(eta, dmu, s0)
    assert x.shape == (1, 1, 2, 16)
    np.testing.assert_allclose(x[0, 0, 0, :6], [1.0, -0.5, 0.2, 0.5, 0.6, 0.0], rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(x[0, 0, 1, :6], [0.0, 2.0, -1.0, 0.25, 0.0, -0.28], rtol=1e-14, atol=1e-15)
    assert not x[..., 6:].any()
    tgt = np.array([[[[0.08, -0.02, 0.0, 0.4], [0.02, 0.16, -0.16, 0.5]]]])
    t = S.residual_target(eta, dmu, s0, tgt)
    np.testing.assert_allclose(t[0, 0, 0, :4], [1.0, 0.0, -0.2, -0.1], rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(t[0, 0, 1, :4], [0.25, 0.0, -1.0, 0.25], rtol=1e-13, atol=1e-15)
    assert not t[..., 4:].any()


def _fp32_gradients(x0_32, params, t32):
    """The network's loss gradient restated in float32 arithmetic (numpy),
    bfloat16 stores at the oracle's points: a stand-in for a float32
    implementation whose only differences from the oracle are roundings."""
    q = lambda a: S.bf16(np.asarray(a, np.float32)).astype(np.float32)
    f = np.float32

    def pad(a):
        N, H, W, C = a.shape
        p = np.zeros((N, H + 2, W + 2, C), f)
        p[:, 1:H + 1, 1:W + 1] = a
        return p

    def conv(x, w, b, relu):
        N, H, W, _ = x.shape
        xp = pad(x)
        y = np.zeros((N, H, W, w.shape[1]), f)
        for a in range(3):
            for c in range(3):
                y += xp[:, a:a + H, c:c + W, :] @ w[3 * a + c].T
        y += b.astype(f)
        return np.maximum(y, f(0)) if relu else y

    layers = S.split_params(params)
    acts = [q(x0_32)]
    for l, (w, b) in enumerate(layers):
        y = conv(acts[-1], q(w), b, l < 3)
        if l < 3:
            acts.append(q(y))
    n = y.shape[0] * y.shape[1] * y.shape[2]
    dy = np.zeros_like(y)
    dy[..., :4] = f(2) * f(1.0 / (4 * n)) * (y - t32)[..., :4]
    dy = q(dy)
    out = [None] * 4
    for l in range(3, -1, -1):
        xp = pad(acts[l])
        N, H, W, _ = acts[l].shape
        gw = np.stack([np.einsum("nhwo,nhwi->oi", dy, xp[:, a:a + H, c:c + W, :]) for a in range(3)
                       for c in range(3)]).astype(f)
        out[l] = (gw, dy.sum(axis=(0, 1, 2), dtype=f))
        if l == 0:
            break
        wq = q(layers[l][0])
        dyp = pad(dy)
        dx = np.zeros(acts[l].shape, f)
        for a in range(3):
            for c in range(3):
                dx += dyp[:, 2 - a:2 - a + H, 2 - c:2 - c + W, :] @ wq[3 * a + c]
        dy = np.where(acts[l] > 0, q(dx), f(0))
    return np.concatenate([np.concatenate([g[0].ravel(), g[1]]) for g in out]).astype(np.float64)


def test_gradient_tolerance_covers_float32_and_rejects_index_mistakes():
    rng = np.random.default_rng(5)
    n, H, W = 2, 12, 40
    params = []
    for l, (ci, co) in enumerate(S.LAYERS):
        used = 6 if l == 0 else ci
        w = rng.normal(size=(9, co, ci)) * np.sqrt(2.0 / (9 * used))
        w[..., used:] = 0.0
        params += [w.ravel(), 0.1 * rng.normal(size=co)]
    params = np.concatenate(params).astype(np.float32)
    x0 = np.zeros((n, H, W, 16))
    x0[..., :6] = rng.normal(size=(n, H, W, 6))
    x0 = np.asarray(x0, np.float32).astype(np.float64)          # float32 features on both sides
    t = np.zeros((n, H, W, 16))
    t[..., :4] = 0.3 * rng.normal(size=(n, H, W, 4))
    t = np.asarray(t, np.float32).astype(np.float64)
    loss, g, tol = SB.oracle_gradients_and_tolerance(x0, params, t)
    g32 = _fp32_gradients(x0.astype(np.float32), params, t.astype(np.float32))
    assert np.all(np.abs(g32 - g) <= tol)
    assert (np.abs(g32 - g) > 0).any()                          # the restatement does round differently
    k = 0
    for ci, co in S.LAYERS:
        w = g[k:k + 9 * ci * co].reshape(9, co, ci)
        tw = tol[k:k + 9 * ci * co].reshape(9, co, ci)
        nz = w != 0
        h = ci // 2 if ci == 32 else 3                          # layer 0: swap the used channels 0..2, 3..5
        swapped = w.copy()
        swapped[..., :h], swapped[..., h:2 * h] = w[..., h:2 * h], w[..., :h]
        assert (np.abs(swapped - w) > tw)[nz].mean() > 0.9
        assert (np.abs(np.roll(w, 1, axis=0) - w) > tw)[nz].mean() > 0.5
        k += 9 * ci * co + co
