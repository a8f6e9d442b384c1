"""Pins of the oracle's inertial source terms (the terms the paper drops by the
assumption of Sec. 4.4; readings R23-R25): the rotational flow field is a
stationary solution of the full PDE, an accelerating camera starts the flow
at -rho a_c, the increment turns at -2 Omega, and an exact-rational restatement
agrees with the C code."""
import numpy as np
import pytest

from tests import hand_stepper as hs


def _pinhole(f, n):
    j = (np.arange(n) + 0.5 - n / 2) / f
    x, y = np.meshgrid(j, j)
    return x, y


@pytest.mark.parametrize("omega", [(0.02, -0.015, 0.01), (-0.01, 0.02, -0.025)])
def test_rotational_flow_is_stationary_with_the_inertial_terms(oracle, omega):
    # A camera rotating at constant Omega (rad/frame) in a static scene sees the
    # structure flow w = -Omega x eta at every ray, for ever: the flow does not
    # depend on depth, and the rays rotate with the camera.  The full PDE
    # (transport, -w<eta,w>, -Omega x w + a_w with a_w = -Omega x (w + Omega x eta))
    # must keep it unchanged; the transport alone moves it by about
    # -Omega x (Omega x eta) per frame.  The one-frame change with the terms
    # refines away at first order in the central window |x|, |y| < 0.025 of
    # the pinhole grid (a wider window keeps the grid's O(x y) inconsistency,
    # reading G2, which does not refine away).
    om = np.asarray(omega)
    rel = []
    for n, f, N in [(96, 80.0, 4), (192, 160.0, 8), (384, 320.0, 16)]:
        eta, B, dmu = oracle.geometry(n, n, f, f, n / 2, n / 2)
        w0 = -np.cross(om, eta)
        rho = 0.1 + 0.05 * eta[..., 0]
        with_terms = oracle.propagate(w0, rho, eta, B, dmu, N, flags=oracle.IMU | oracle.SOURCE_SPLIT,
                                      imu=np.concatenate([om, np.zeros(3)]))
        without = oracle.propagate(w0, rho, eta, B, dmu, N, flags=oracle.SOURCE_SPLIT)
        assert with_terms[4] <= 1.0
        x, y = _pinhole(f, n)
        core = (np.abs(x) < 0.025) & (np.abs(y) < 0.025)
        e_with = np.abs(with_terms[0] - w0)[core].max()
        e_without = np.abs(without[0] - w0)[core].max()
        # the transport alone: about |Omega x (Omega x eta)| per frame
        ref = np.abs(np.cross(om, np.cross(om, eta)))[core].max()
        assert 0.5 * ref < e_without < 2.0 * ref
        rel.append(e_with / e_without)
    assert rel[0] < 0.1
    assert 0.4 < rel[1] / rel[0] < 0.6 and 0.4 < rel[2] / rel[1] < 0.6, rel


def test_accelerating_camera_starts_the_flow_at_minus_rho_a(oracle):
    # Camera at rest at t = 0 with linear acceleration a (Omega = 0) in front of
    # a static fronto-parallel plane at depth Z: v_c(t) = a t, so the structure
    # flow rho (v_p - v_c) is -rho a t, i.e. -rho a dt^2 after one frame in
    # frame units (a_f = a dt^2), up to O(a_f^2) from the transport of the
    # growing flow and from the plane's approach (reading R24: -rho a_c).
    n, f, N, Z = 64, 40.0, 2, 3.0
    eta, B, dmu = oracle.geometry(n, n, f, f, n / 2, n / 2)
    rho = eta[..., 2] / Z
    errs = []
    for scale in (1.0, 0.5):
        a_f = scale * np.array([0.002, -0.001, 0.003])
        w, _, r, _, _ = oracle.propagate(np.zeros((n, n, 3)), rho, eta, B, dmu, N, flags=oracle.IMU,
                                         imu=np.concatenate([np.zeros(3), a_f]))
        truth = -rho[..., None] * a_f
        assert (np.einsum("hwc,c->hw", w, a_f) < 0).all()
        errs.append(np.abs(w - truth).max() / np.abs(truth).max())
    # relative error O(a_f): the absolute error is second order in a_f
    assert errs[0] < 1e-2
    assert 0.4 < errs[1] / errs[0] < 0.6, errs
    # without the terms the flow stays zero (the paper's assumption)
    w0 = oracle.propagate(np.zeros((n, n, 3)), rho, eta, B, dmu, N)[0]
    assert not w0.any()


def test_increment_turns_at_minus_two_omega(oracle):
    # Lower levels: under the stationary rotational flow w = -Omega x eta
    # (<eta, w> = 0, so no -dw<eta,w> source) a uniform increment dw is not
    # moved by the transport and obeys d(dw)/dt = -2 Omega x dw, a rotation by
    # -2 |Omega| about Omega per frame; N explicit Euler steps converge to it at
    # first order.  (Checked away from the image border, where the replicated
    # neighbours keep w from being exactly stationary.)
    n = 32
    eta, B, dmu = oracle.geometry(n, n, 24.0, 24.0, n / 2, n / 2)
    om = np.array([0.03, -0.02, 0.05])
    d0 = np.array([0.004, 0.001, -0.002])
    th = 2 * np.linalg.norm(om); k = om / np.linalg.norm(om)
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    R = np.eye(3) - np.sin(th) * K + (1 - np.cos(th)) * K @ K      # rotation by -th about k
    errs = []
    for N in (4, 8, 16):
        _, dw, _, _, _ = oracle.propagate(-np.cross(om, eta), np.ones((n, n)), eta, B, dmu, N,
                                          dw=np.tile(d0, (n, n, 1)), Y=np.zeros((n, n)), flags=oracle.IMU,
                                          imu=np.concatenate([om, np.zeros(3)]))
        c = slice(n // 2 - 4, n // 2 + 4)
        errs.append(np.abs(dw[c, c] - R @ d0).max() / np.abs(d0).max())
    assert errs[0] < 0.01
    assert 0.4 < errs[1] / errs[0] < 0.6 and 0.4 < errs[2] / errs[1] < 0.6, errs


@pytest.mark.parametrize("mode", ["top", "lower"])
def test_inertial_step_matches_exact_rational_hand_stepper(oracle, mode):
    rng = np.random.default_rng(11)
    H, W, N = 5, 6, 2
    eta, B, dmu = oracle.geometry(H, W, 5.0, 5.0, 3.1, 2.2)
    w = rng.uniform(-0.5, 0.5, (H, W, 3)) * dmu[..., None]
    rho = rng.uniform(0.2, 1.0, (H, W))
    dw = rng.uniform(-0.2, 0.2, (H, W, 3)) * dmu[..., None] if mode == "lower" else None
    Y = rng.uniform(size=(H, W)) if mode == "lower" else None
    imu = np.array([0.03, -0.05, 0.02, 0.004, -0.002, 0.003])
    got = oracle.propagate(w, rho, eta, B, dmu, N, dw=dw, Y=Y, flags=oracle.IMU, imu=imu)
    F = hs.to_fr
    ew, er, ed, ey = hs.propagate(H, W, N, F(eta), F(B[:, :, 0]), F(B[:, :, 1]), F(dmu), F(w), F(rho),
                                  dw=None if dw is None else F(dw), Y=None if Y is None else F(Y),
                                  imu=(F(imu[:3]), F(imu[3:])))
    np.testing.assert_allclose(got[0], hs.to_float(ew), rtol=0, atol=1e-15)
    np.testing.assert_allclose(got[2], hs.to_float(er), rtol=0, atol=1e-14)
    if dw is not None:
        np.testing.assert_allclose(got[1], hs.to_float(ed), rtol=0, atol=1e-15)
