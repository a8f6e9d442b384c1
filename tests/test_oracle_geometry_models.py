"""Pins of the oracle's grid geometry and measurement models (CPU only).

Each expected value comes from a closed form, an invariant or a library
routine applied to the definition -- never from the oracle itself.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ---------------------------------------------------------------- geometry

def test_basis_orthonormal_and_tangent(oracle):
    eta, B, dmu = oracle.geometry(24, 40, 30.0, 25.0, 21.0, 11.5)
    np.testing.assert_allclose(np.linalg.norm(eta, axis=-1), 1.0, atol=1e-14)
    gram = np.einsum("hwac,hwbc->hwab", B, B)
    np.testing.assert_allclose(gram, np.broadcast_to(np.eye(2), gram.shape), atol=1e-14)
    np.testing.assert_allclose(np.einsum("hwac,hwc->hwa", B, eta), 0.0, atol=1e-13)
    assert (dmu > 0).all()


def test_spacing_closed_form_on_principal_row(oracle):
    # cy chosen so row 4 passes through the principal point (y = 0): rays lie in
    # the x-z plane at angles atan(x); dmu = sin(angle between neighbours),
    # b1 = d eta / d theta = (cos t, 0, -sin t), b2 = e_y.
    H, W, f, cx, cy = 10, 16, 8.0, 8.0, 4.5
    eta, B, dmu = oracle.geometry(H, W, f, f, cx, cy)
    j = np.arange(W)
    t0 = np.arctan((j + 0.5 - cx) / f)
    t1 = np.arctan((j + 1.5 - cx) / f)
    np.testing.assert_allclose(dmu[4], np.sin(t1 - t0), rtol=1e-13)
    np.testing.assert_allclose(B[4, :, 0], np.stack([np.cos(t0), 0 * t0, -np.sin(t0)], -1), atol=1e-14)
    np.testing.assert_allclose(B[4, :, 1], np.broadcast_to([0.0, 1.0, 0.0], (W, 3)), atol=1e-14)


def test_basis_orientation_follows_columns_and_rows(oracle):
    eta, B, dmu = oracle.geometry(12, 12, 9.0, 9.0, 6.0, 6.0)
    dcol = eta[:, 1:] - eta[:, :-1]
    drow = eta[1:] - eta[:-1]
    assert (np.einsum("hwc,hwc->hw", B[:, :-1, 0], dcol) > 0).all()
    assert (np.einsum("hwc,hwc->hw", B[:-1, :, 1], drow) > 0).all()


def test_level_intrinsics_put_rays_through_block_centres(oracle):
    fx, fy, cx, cy = 40.0, 36.0, 33.0, 30.0
    eta2, _, _ = oracle.geometry(16, 16, *oracle.level_intrinsics(fx, fy, cx, cy, 2))
    i, j = np.meshgrid(np.arange(16), np.arange(16), indexing="ij")
    # centre of the 2x2 block of level-1 pixels (2i..2i+1, 2j..2j+1) is the
    # level-1 continuous coordinate (2j + 1, 2i + 1)
    d = np.stack([(2 * j + 1 - cx) / fx, (2 * i + 1 - cy) / fy, np.ones_like(i, float)], -1)
    np.testing.assert_allclose(eta2, d / np.linalg.norm(d, axis=-1, keepdims=True), atol=1e-15)


# ---------------------------------------------------------------- image model (Eqs. 30-31)

def _flat_geom(H, W):
    B = np.zeros((H, W, 2, 3)); B[..., 0, 0] = 1.0; B[..., 1, 1] = 1.0
    eta = np.zeros((H, W, 3)); eta[..., 2] = 1.0
    return eta, B, np.ones((H, W))


def test_image_model_constant(oracle):
    eta, B, dmu = oracle.geometry(12, 14, 10.0, 10.0, 7.0, 6.0)
    Yhat, db, g = oracle.image_model(np.full((12, 14), 0.37), B, dmu)
    np.testing.assert_allclose(Yhat, 0.37, atol=1e-15)
    np.testing.assert_allclose(db, 0.0, atol=1e-15)
    np.testing.assert_allclose(g, 0.0, atol=1e-15)


def test_image_model_linear_ramp_exact_in_interior(oracle):
    H, W = 14, 17
    i, j = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    Y = 0.2 + 0.03 * j - 0.05 * i
    _, B, dmu = _flat_geom(H, W)
    Yhat, db, _ = oracle.image_model(Y, B, dmu)
    sl = np.s_[2:-2, 2:-2]
    np.testing.assert_allclose(Yhat[sl], Y[sl], atol=1e-14)
    np.testing.assert_allclose(db[sl][..., 0], 0.03, atol=1e-14)   # slope along columns (beta_1)
    np.testing.assert_allclose(db[sl][..., 1], -0.05, atol=1e-14)  # slope along rows (beta_2)


def test_image_model_quadratics(oracle):
    # sum_d g(d) d^2 = 1 for g = [1,4,6,4,1]/16, so the fitted constant of j^2 is
    # j^2 + 1 and its slope 2j; for i*j the constant is i*j, slopes (i, j).
    H, W = 13, 15
    i, j = np.meshgrid(np.arange(H, dtype=float), np.arange(W, dtype=float), indexing="ij")
    _, B, dmu = _flat_geom(H, W)
    sl = np.s_[2:-2, 2:-2]
    Yhat, db, _ = oracle.image_model(j ** 2, B, dmu)
    np.testing.assert_allclose(Yhat[sl], (j ** 2 + 1)[sl], atol=1e-12)
    np.testing.assert_allclose(db[sl][..., 0], (2 * j)[sl], atol=1e-12)
    np.testing.assert_allclose(db[sl][..., 1], 0.0, atol=1e-12)
    Yhat, db, _ = oracle.image_model(i * j, B, dmu)
    np.testing.assert_allclose(Yhat[sl], (i * j)[sl], atol=1e-12)
    np.testing.assert_allclose(db[sl][..., 0], i[sl], atol=1e-12)
    np.testing.assert_allclose(db[sl][..., 1], j[sl], atol=1e-12)


def test_image_model_matches_weighted_lstsq_with_replicated_border(oracle):
    rng = np.random.default_rng(5)
    H, W = 9, 11
    Y = rng.uniform(size=(H, W))
    _, B, dmu = _flat_geom(H, W)
    Yhat, db, _ = oracle.image_model(Y, B, dmu)
    g = np.array([1, 4, 6, 4, 1]) / 16.0
    for (pi, pj) in [(0, 0), (0, 5), (4, 10), (8, 8), (4, 5), (1, 9)]:
        rows, rhs, wts = [], [], []
        for di in range(-2, 3):
            for dj in range(-2, 3):
                qi, qj = min(max(pi + di, 0), H - 1), min(max(pj + dj, 0), W - 1)
                rows.append([1.0, dj, di]); rhs.append(Y[qi, qj]); wts.append(g[di + 2] * g[dj + 2])
        sw = np.sqrt(np.array(wts))
        x = np.linalg.lstsq(np.array(rows) * sw[:, None], np.array(rhs) * sw, rcond=None)[0]
        np.testing.assert_allclose([Yhat[pi, pj], db[pi, pj, 0], db[pi, pj, 1]], x, atol=1e-13)


@pytest.mark.parametrize("which", ["image", "invdepth"])
def test_lifted_gradient_is_dmu_squared_times_sphere_gradient(oracle, which):
    # For a field F(eta) = <k, eta> the gradient on the sphere is P k.  The lift
    # dmu * B * d_beta (reading R4) equals dmu^2 times it to O(dmu); with
    # B^T instead of B, or a missing dmu, this fails by orders of magnitude.
    H = W = 21
    f = 200.0
    eta, B, dmu = oracle.geometry(H, W, f, f, W / 2, H / 2)
    k = np.array([0.7, -0.4, 0.3])
    F = eta @ k
    if which == "image":
        _, _, g = oracle.image_model(F, B, dmu)
    else:
        _, g = oracle.invdepth_model(F, np.ones((H, W), np.uint8), B, dmu)
    Pk = k - eta * (eta @ k)[..., None]
    sl = np.s_[4:-4, 4:-4]
    ratio = g[sl] / dmu[sl][..., None] ** 2
    np.testing.assert_allclose(ratio, Pk[sl], rtol=0, atol=2e-2 * np.abs(Pk).max())
    np.testing.assert_allclose(np.einsum("hwc,hwc->hw", g, eta), 0.0, atol=1e-15)


# ---------------------------------------------------------------- inverse-depth model (Eqs. 32-34)

def test_invdepth_step_edge_gives_zero_gradient(oracle):
    H, W = 6, 16
    rho = np.where(np.arange(W) < 8, 1.0, 2.0)[None, :].repeat(H, 0)
    _, B, dmu = _flat_geom(H, W)
    db, g = oracle.invdepth_model(rho, np.ones((H, W), np.uint8), B, dmu)
    np.testing.assert_array_equal(db, 0.0)   # min-abs picks the flat side on both edge pixels


def test_invdepth_ramp_and_border(oracle):
    H, W = 7, 9
    i, j = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    rho = 1.0 + 0.125 * j + 0.0625 * i
    _, B, dmu = _flat_geom(H, W)
    db, _ = oracle.invdepth_model(rho, np.ones((H, W), np.uint8), B, dmu)
    np.testing.assert_array_equal(db[1:-1, 1:-1, 0], 0.125)
    np.testing.assert_array_equal(db[1:-1, 1:-1, 1], 0.0625)
    # replicated border: one side difference is 0 and has the smaller magnitude
    np.testing.assert_array_equal(db[:, 0, 0], 0.0)
    np.testing.assert_array_equal(db[:, -1, 0], 0.0)
    np.testing.assert_array_equal(db[0, :, 1], 0.0)
    np.testing.assert_array_equal(db[-1, :, 1], 0.0)


def test_invdepth_tie_takes_forward_difference(oracle):
    W = 11
    rho = np.abs(np.arange(W) - 5.0)[None, :].repeat(3, 0) + 1.0
    _, B, dmu = _flat_geom(3, W)
    db, _ = oracle.invdepth_model(rho, np.ones((3, W), np.uint8), B, dmu)
    assert db[1, 5, 0] == 1.0      # |d+| = |d-| = 1 -> forward difference (+1)


def test_invdepth_missing_measurements(oracle):
    H, W = 5, 8
    rho = np.tile(np.arange(W, dtype=float) * 0.5 + 1.0, (H, 1))
    rho[:, 3] = 9.0      # outlier column that will be marked invalid
    valid = np.ones((H, W), np.uint8); valid[:, 3] = 0
    _, B, dmu = _flat_geom(H, W)
    db, g = oracle.invdepth_model(rho, valid, B, dmu)
    np.testing.assert_array_equal(db[:, 3], 0.0)                 # no measurement at the pixel
    np.testing.assert_array_equal(db[1:-1, 2, 0], 0.5)           # right side missing -> backward
    np.testing.assert_array_equal(db[1:-1, 4, 0], 0.5)           # left side missing -> forward
    valid2 = valid.copy(); valid2[:, 5] = 0
    db2, _ = oracle.invdepth_model(rho, valid2, B, dmu)
    np.testing.assert_array_equal(db2[:, 4, 0], 0.0)             # both sides missing -> 0
