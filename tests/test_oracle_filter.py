"""Pins of the oracle's whole predictor-update loop (Sec. 4, Fig. 3)."""
import numpy as np
import pytest

from paper_2406_18031_b300 import scenes


def _filter(oracle, H, W, L, iters, smooth, **kw):
    p = oracle.Params(fx=W / 2.0, fy=W / 2.0, cx=W / 2.0, cy=H / 2.0, iters=iters, smooth=smooth, **kw)
    return oracle.Filter(H, W, L, p)


def test_first_frame_initialises_only(oracle):
    # R18: zero flow, inverse depth = lambda_ref / lambda, no measurement -> 0
    rng = np.random.default_rng(0)
    H = W = 32
    f = _filter(oracle, H, W, 2, [2, 1], [2, 4], lambda_ref=2.0)
    img = rng.uniform(size=(H, W)); lam = rng.uniform(1, 5, size=(H, W)); lam[3, 4] = -1.0; lam[5, 6] = np.inf
    flow, inv = f.step(img, lam, 1 / 600)
    np.testing.assert_array_equal(flow, 0.0)
    expect = np.where(np.isfinite(lam) & (lam > 0), 2.0 / lam, 0.0)
    np.testing.assert_allclose(inv, expect, rtol=1e-15)


def test_zero_motion_keeps_zero_flow(oracle):
    # static image and depth: every temporal term vanishes, so the flow stays
    # exactly zero at every level and the inverse depth stays at rho-hat
    rng = np.random.default_rng(1)
    H = W = 32
    img = rng.uniform(size=(H, W)); lam = rng.uniform(1, 5, size=(H, W))
    f = _filter(oracle, H, W, 3, [3, 2, 1], [2, 4, 4])
    for _ in range(6):
        flow, inv = f.step(img, lam, 1 / 300)
        np.testing.assert_array_equal(flow, 0.0)
        np.testing.assert_allclose(inv, 1.0 / lam, rtol=1e-14)
    for h in range(3):
        s = f.get_state(h)
        np.testing.assert_array_equal(s["w"], 0.0)
        np.testing.assert_array_equal(s["dw"], 0.0)


def test_frame_time_change_rescales_the_state(oracle):
    # R9: the state is rad/frame; a new dt scales w and dw by dt_new / dt_old
    seq = scenes.plane64(frames=3)
    a = _filter(oracle, 64, 64, 2, [2, 1], [2, 4])
    b = _filter(oracle, 64, 64, 2, [2, 1], [2, 4])
    rng = np.random.default_rng(2)
    for h in range(2):
        n = 64 >> h
        w = rng.normal(size=(n, n, 3)) * 1e-3; dw = rng.normal(size=(n, n, 3)) * 1e-4
        r = rng.uniform(0.1, 0.3, size=(n, n)); y = rng.uniform(size=(n, n))
        a.set_state(h, w=w, dw=dw, rho=r, Yhat=y, dt_prev=2.0 * seq.dt)
        b.set_state(h, w=0.5 * w, dw=0.5 * dw, rho=r, Yhat=y, dt_prev=seq.dt)
    fa, ia = a.step(seq.image[1], seq.range[1], seq.dt)
    fb, ib = b.step(seq.image[1], seq.range[1], seq.dt)
    np.testing.assert_allclose(fa, fb, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(ia, ib, rtol=1e-13)


def test_plane_sequence_approaches_the_closed_form_flow(oracle):
    # config "plane64": the closed-form structure flow is w = -v eta_z / Z(t).
    # Starting from zero (R18) the filter's error shrinks frame after frame.
    seq = scenes.plane64(frames=20)
    f = _filter(oracle, 64, 64, 1, [2], [2])
    eta, _, dmu = f.geometry(0)
    errs = []
    for k in range(seq.frames):
        flow, _ = f.step(seq.image[k], seq.range[k], seq.dt)
        Z = seq.meta["depth"] - seq.v[k, 2] * k * seq.dt
        w_gt = -seq.v[k][:, None, None] * eta[..., 2][None] / Z
        errs.append(np.mean(np.linalg.norm(flow - w_gt, axis=0) * seq.dt / dmu))
    assert errs[1] < errs[0] and errs[-1] < 0.85 * errs[0]
    assert all(b <= a + 1e-12 for a, b in zip(errs[1:], errs[2:]))


def test_invalid_configurations_are_rejected(oracle):
    with pytest.raises(ValueError):
        _filter(oracle, 30, 30, 3, [1, 1, 1], [2, 4, 4])   # 30 not divisible by 4
