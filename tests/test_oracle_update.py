"""Pins of the oracle's update, blend, smoothing and pyramid (Sec. 4.5, Eq. 26)."""
import numpy as np
import pytest


def _plane_case(n=64, f=64.0, Z0=4.0, v=(1.0, 0.5, 1.0), dt=1 / 30):
    """Two exact frames of a textured fronto-parallel plane under camera
    translation, with the exact structure flow (rad/frame) and inverse depth."""
    import oracle
    eta, B, dmu = oracle.geometry(n, n, f, f, n / 2, n / 2)
    v = np.asarray(v)

    def tex(X, Y):
        return 0.5 + 0.2 * np.sin(3.1 * X + 0.3) * np.cos(2.3 * Y - 0.2) + 0.1 * np.sin(5.3 * X - 4.1 * Y)

    def render(t):
        c = v * t
        lam = (Z0 - c[2]) / eta[..., 2]
        P = c + lam[..., None] * eta
        return tex(P[..., 0], P[..., 1]), 1.0 / lam

    Y0, r0 = render(0.0)
    Y1, r1 = render(dt)
    w = -v[None, None, :] * eta[..., 2:3] / (Z0 - v[2] * dt / 2) * dt
    return eta, B, dmu, Y0, r0, Y1, r1, w


def _inputs(oracle, case):
    eta, B, dmu, Y0, r0, Y1, r1, w = case
    n = Y0.shape[0]
    valid = np.ones((n, n), np.uint8)
    Yh0, _, _ = oracle.image_model(Y0, B, dmu)
    Yh1, _, gY = oracle.image_model(Y1, B, dmu)
    _, gR = oracle.invdepth_model(r1, valid, B, dmu)
    return eta, dmu, Yh0, Yh1, gY, r0, r1, gR, valid, w


def test_no_data_weight_returns_the_prior(oracle):
    rng = np.random.default_rng(0)
    H, W = 5, 6
    eta, B, dmu = oracle.geometry(H, W, 5.0, 5.0, 3.0, 2.5)
    prior = rng.normal(size=(H, W, 3))
    x = oracle.update((0.0, 0.0, 0.3), eta, dmu, rng.uniform(size=(H, W)), rng.normal(size=(H, W, 3)),
                      rng.uniform(size=(H, W)), rng.normal(size=(H, W, 3)), np.ones((H, W), np.uint8),
                      rng.uniform(size=(H, W)), rng.uniform(size=(H, W)), prior)
    np.testing.assert_allclose(x, prior, rtol=1e-15)


def test_missing_depth_drops_the_depth_term(oracle):
    rng = np.random.default_rng(1)
    H, W = 4, 7
    eta, B, dmu = oracle.geometry(H, W, 6.0, 6.0, 3.5, 2.0)
    a = [rng.uniform(size=(H, W)), rng.normal(size=(H, W, 3)) * 0.01, rng.uniform(size=(H, W)),
         rng.normal(size=(H, W, 3)) * 0.01]
    rest = [rng.uniform(size=(H, W)), rng.uniform(size=(H, W)), rng.normal(size=(H, W, 3)) * 0.01]
    no_meas = oracle.update((1.0, 1.0, 1e-3), eta, dmu, *a, np.zeros((H, W), np.uint8), *rest)
    no_gain = oracle.update((1.0, 0.0, 1e-3), eta, dmu, *a, np.ones((H, W), np.uint8), *rest)
    np.testing.assert_array_equal(no_meas, no_gain)


def test_solution_is_stationary_point_of_the_cost(oracle):
    # d/dx [g1 E_Y^2 + g2 E_rho^2 + g3 |x - prior|^2] = 0 with the E terms of
    # Eqs. 43-45 (reading R6), evaluated by central finite differences of the
    # cost itself.
    rng = np.random.default_rng(2)
    H, W = 3, 4
    eta, B, dmu = oracle.geometry(H, W, 4.0, 4.0, 2.0, 1.5)
    Yh, Yr = rng.uniform(size=(H, W)), rng.uniform(size=(H, W))
    gY = np.einsum("hwkc,hwk->hwc", B, rng.normal(size=(H, W, 2))) * 0.3
    gR = np.einsum("hwkc,hwk->hwc", B, rng.normal(size=(H, W, 2))) * 0.3
    rh, rr = rng.uniform(0.2, 1, size=(H, W)), rng.uniform(0.2, 1, size=(H, W))
    prior = rng.normal(size=(H, W, 3)) * 0.1
    g = (0.7, 1.3, 0.05)
    x = oracle.update(g, eta, dmu, Yh, gY, rh, gR, np.ones((H, W), np.uint8), Yr, rr, prior)

    def cost(p, xx):
        e, d2 = eta[p], dmu[p] ** 2
        P = np.eye(3) - np.outer(e, e)
        EY = gY[p] @ P @ xx + d2 * (Yh[p] - Yr[p])
        ER = gR[p] @ P @ xx + d2 * ((rh[p] - rr[p]) + rh[p] * (e @ xx))
        Et = xx - prior[p]
        return g[0] * EY ** 2 + g[1] * ER ** 2 + g[2] * Et @ Et

    h = 1e-6
    for p in np.ndindex(H, W):
        grad = [(cost(p, x[p] + h * np.eye(3)[c]) - cost(p, x[p] - h * np.eye(3)[c])) / (2 * h) for c in range(3)]
        np.testing.assert_allclose(grad, 0.0, atol=1e-8)


def test_ground_truth_is_nearly_a_fixed_point(oracle):
    # Exact data from a moving plane: with the true structure flow as prior, the
    # brightness (Eq. 43) and inverse-depth (Eq. 44) residuals vanish to first
    # order, so the update barely moves it.  Reversing the time order of the
    # data (a sign error in the temporal terms) moves it by a large fraction.
    eta, dmu, Yh0, Yh1, gY, r0, r1, gR, valid, w = _inputs(oracle, _plane_case())
    g3 = 1e-4 * dmu[32, 32] ** 2
    core = np.s_[8:-8, 8:-8]
    x = oracle.update((1.0, 1.0, g3), eta, dmu, Yh1, gY, r1, gR, valid, Yh0, r0, w)
    rel = np.linalg.norm(x - w, axis=-1) / np.linalg.norm(w, axis=-1)
    assert np.median(rel[core]) < 0.05
    xs = oracle.update((1.0, 1.0, g3), eta, dmu, Yh0, gY, r0, gR, valid, Yh1, r1, w)
    rels = np.linalg.norm(xs - w, axis=-1) / np.linalg.norm(w, axis=-1)
    assert np.median(rels[core]) > 0.3


def test_depth_term_recovers_the_normal_component(oracle):
    # With only the inverse-depth term (g1 = 0), a prior that is wrong along the
    # viewing ray (normal flow, Sec. 4.5) is pulled back to the truth: E_rho
    # constrains <eta, w> through the rho-hat <eta, w> term of Eq. 44.  The
    # depth row is O(dmu^2 rho) while the prior weight is g3, so g2 is raised
    # until the depth term dominates the prior.
    eta, dmu, Yh0, Yh1, gY, r0, r1, gR, valid, w = _inputs(oracle, _plane_case())
    g3 = 1e-4 * dmu[32, 32] ** 2
    pert = 0.5 * np.linalg.norm(w, axis=-1, keepdims=True) * eta
    x = oracle.update((0.0, 1e3, g3), eta, dmu, Yh1, gY, r1, gR, valid, Yh0, r0, w + pert)
    core = np.s_[8:-8, 8:-8]
    left = np.einsum("hwc,hwc->hw", x - w, eta)[core]
    # one row a + dmu^2 rho eta removes the error along itself; what stays is
    # the fraction |a|^2 / |row|^2 of the normal error (about 7% here)
    assert np.median(np.abs(left) / np.linalg.norm(pert, axis=-1)[core]) < 0.12


def test_blend_closed_form(oracle):
    rh = np.array([0.5, 0.25, 1.0]); rp = np.array([0.3, 0.5, 0.2]); valid = np.array([1, 1, 0], np.uint8)
    out = oracle.blend(3.0, 1.0, rh, valid, rp)
    np.testing.assert_allclose(out, [(3 * 0.5 + 0.3) / 4, (3 * 0.25 + 0.5) / 4, 0.2], rtol=1e-15)
    np.testing.assert_array_equal(oracle.blend(0.0, 1.0, rh, np.ones(3, np.uint8), rp), rp)
    np.testing.assert_array_equal(oracle.blend(1.0, 0.0, rh, np.ones(3, np.uint8), rp), rh)


def test_smoothing_impulse_response_and_linear_fields(oracle):
    H, W = 21, 23
    f = np.zeros((H, W, 3)); f[10, 11, 1] = 625.0
    s1 = oracle.smooth(f, 1)
    expect1 = np.zeros((H, W)); expect1[8:13, 9:14] = 25.0
    np.testing.assert_allclose(s1[..., 1], expect1, atol=1e-12)
    s2 = oracle.smooth(f, 2)
    t = 5.0 - np.abs(np.arange(-4, 5))       # box * box = triangle [1..5..1]
    expect2 = np.zeros((H, W)); expect2[6:15, 7:16] = np.outer(t, t)
    np.testing.assert_allclose(s2[..., 1], expect2, atol=1e-12)
    np.testing.assert_array_equal(s2[..., 0], 0.0)
    i, j = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    lin = np.stack([0.1 * i + 0.2 * j, -0.3 * j, np.full((H, W), 0.7)], -1)
    s = oracle.smooth(lin, 2)
    np.testing.assert_allclose(s[4:-4, 4:-4], lin[4:-4, 4:-4], atol=1e-13)


def test_pyramid_down(oracle):
    Y = np.arange(16.0).reshape(4, 4)
    rho = np.arange(1.0, 17.0).reshape(4, 4)
    valid = np.ones((4, 4), np.uint8); valid[0, 0] = 0; valid[2:, 2:] = 0
    Y2, r2, v2 = oracle.downsample(Y, rho, valid)
    np.testing.assert_array_equal(Y2, [[2.5, 4.5], [10.5, 12.5]])
    np.testing.assert_array_equal(r2, [[(2 + 5 + 6) / 3, (3 + 4 + 7 + 8) / 4], [(9 + 10 + 13 + 14) / 4, 0.0]])
    np.testing.assert_array_equal(v2, [[1, 1], [1, 0]])


def test_pyramid_up_is_bilinear_at_pixel_centres(oracle):
    Hc, Wc = 6, 7
    I, J = np.meshgrid(np.arange(Hc), np.arange(Wc), indexing="ij")
    wc = np.stack([1.0 + 0.5 * I - 0.25 * J, 2.0 * J, np.full((Hc, Wc), 3.0)], -1)
    dw = np.full((2 * Hc, 2 * Wc, 3), 0.125)
    out = oracle.upsample_add(wc, dw)
    i, j = np.meshgrid(np.arange(2 * Hc), np.arange(2 * Wc), indexing="ij")
    ci, cj = (i + 0.5) / 2 - 0.5, (j + 0.5) / 2 - 0.5    # fine centre in coarse pixel units
    expect = np.stack([1.0 + 0.5 * ci - 0.25 * cj, 2.0 * cj, np.full(ci.shape, 3.0)], -1) + 0.125
    np.testing.assert_allclose(out[1:-1, 1:-1], expect[1:-1, 1:-1], atol=1e-14)
    # replicated border: the outermost fine pixels see the edge coarse value
    np.testing.assert_allclose(out[0, 0], wc[0, 0] + 0.125, atol=1e-14)
    np.testing.assert_allclose(out[-1, -1], wc[-1, -1] + 0.125, atol=1e-14)
