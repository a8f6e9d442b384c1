"""Pins of the oracle's remapping of camera data onto the filter's grid
(readings R26, R27): identities and exact permutations for the pinhole path,
second-order convergence to an analytic panorama, nearest-pixel containment
for range, no seam at the longitude wrap, and no measurement out of view."""
import numpy as np
import pytest


def _img(rng, H, W):
    return rng.uniform(size=(H, W))


def _Rx(a):
    c, s = np.cos(a), np.sin(a)
    return np.array([[1, 0, 0], [0, c, -s], [0, s, c]])


def _Ry(a):
    c, s = np.cos(a), np.sin(a)
    return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]])


def test_pinhole_identity_returns_the_frame(oracle):
    rng = np.random.default_rng(1)
    H, W = 24, 40
    img, lam = _img(rng, H, W), rng.uniform(1, 9, size=(H, W))
    K = (31.0, 29.0, 19.5, 12.25)
    oi, orng = oracle.remap_pinhole(H, W, K, np.eye(3), K, img, lam)
    # the centre maps back onto the centre up to rounding of (j + 1/2 - c)/f
    np.testing.assert_allclose(oi, img, rtol=0, atol=1e-12)
    np.testing.assert_array_equal(orng, lam)


def test_pinhole_principal_point_shift_is_a_pixel_shift(oracle):
    # the camera's principal point 3 px to the right: grid column j sees camera
    # column j + 3 at its centre; columns beyond the frame are out of view
    rng = np.random.default_rng(2)
    H, W = 20, 30
    img, lam = _img(rng, H, W), rng.uniform(1, 9, size=(H, W))
    oi, orng = oracle.remap_pinhole(H, W, (25.0, 25.0, 15.0, 10.0), np.eye(3), (25.0, 25.0, 18.0, 10.0), img, lam)
    np.testing.assert_allclose(oi[:, :W - 3], img[:, 3:], rtol=0, atol=1e-12)
    np.testing.assert_array_equal(orng[:, :W - 3], lam[:, 3:])
    assert not oi[:, W - 2:].any() and not orng[:, W - 2:].any()


def test_pinhole_quarter_turn_is_a_transpose_flip(oracle):
    # R = rotation by 90 degrees about the optical axis (camera <- grid): the
    # ray (x, y, 1) of the grid is (-y, x, 1) for the camera, so grid pixel
    # (i, j) is camera pixel (j, n - 1 - i) exactly
    rng = np.random.default_rng(3)
    n = 17
    img, lam = _img(rng, n, n), rng.uniform(1, 9, size=(n, n))
    R = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    K = (12.0, 12.0, n / 2, n / 2)
    oi, orng = oracle.remap_pinhole(n, n, K, R, K, img, lam)
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    np.testing.assert_allclose(oi, img[j, n - 1 - i], rtol=0, atol=1e-12)
    np.testing.assert_array_equal(orng, lam[j, n - 1 - i])


def test_pinhole_rays_behind_the_camera_have_no_measurement(oracle):
    rng = np.random.default_rng(4)
    img, lam = _img(rng, 16, 16), rng.uniform(1, 9, size=(16, 16))
    oi, orng = oracle.remap_pinhole(16, 16, (8.0, 8.0, 8.0, 8.0), _Ry(np.pi), (8.0, 8.0, 8.0, 8.0), img, lam)
    assert not oi.any() and not orng.any()


def _pano_function(d):
    return 0.5 + 0.3 * np.sin(3.0 * d[..., 0] + 2.0 * d[..., 1]) * np.cos(2.0 * d[..., 2])


def _pano(Hs, Ws):
    """Panorama of the analytic function of direction, sampled at pixel centres."""
    u = (np.arange(Ws) + 0.5) / Ws * 2 * np.pi - np.pi
    v = np.pi / 2 - (np.arange(Hs) + 0.5) / Hs * np.pi
    phi, th = np.meshgrid(u, v)
    d = np.stack([np.cos(th) * np.sin(phi), -np.sin(th), np.cos(th) * np.cos(phi)], -1)
    return _pano_function(d)


def _grid_dirs(n, K, R):
    j = (np.arange(n) + 0.5 - K[2]) / K[0]
    i = (np.arange(n) + 0.5 - K[3]) / K[1]
    x, y = np.meshgrid(j, i)
    m = np.stack([x, y, np.ones_like(x)], -1) @ np.asarray(R).T
    return m / np.linalg.norm(m, axis=-1, keepdims=True)


@pytest.mark.parametrize("R", [np.eye(3), _Ry(np.pi) @ _Rx(0.3)], ids=["forward", "backward_tilted"])
def test_equirect_converges_at_second_order(oracle, R):
    # bilinear interpolation of a smooth panorama: the error to the analytic
    # function at the grid rays falls ~4x per doubling of the panorama; the
    # backward view straddles the longitude wrap (no seam)
    n, K = 48, (24.0, 24.0, 24.0, 24.0)
    truth = _pano_function(_grid_dirs(n, K, R))
    errs = []
    for Hs in (256, 512, 1024):
        oi, _ = oracle.remap_equirect(n, n, K, R, _pano(Hs, 2 * Hs))
        errs.append(np.abs(oi - truth).max())
    assert errs[0] < 1e-3
    assert 0.2 < errs[1] / errs[0] < 0.3 and 0.2 < errs[2] / errs[1] < 0.3, errs


def test_equirect_range_is_the_containing_pixel(oracle):
    # every panorama pixel carries its own id; the remapped range must be the id
    # of the pixel whose longitude-latitude cell contains the grid ray
    Hs, Ws, n, K = 90, 180, 32, (20.0, 20.0, 16.0, 16.0)
    R = _Ry(2.9) @ _Rx(-0.4)
    ids = np.arange(Hs * Ws, dtype=np.float64).reshape(Hs, Ws)
    _, orng = oracle.remap_equirect(n, n, K, R, np.zeros((Hs, Ws)), ids)
    d = _grid_dirs(n, K, R)
    row, col = orng.astype(int) // Ws, orng.astype(int) % Ws
    lon = np.arctan2(d[..., 0], d[..., 2]); lat = np.arcsin(-d[..., 1])
    lo_lon = col / Ws * 2 * np.pi - np.pi; hi_lon = (col + 1) / Ws * 2 * np.pi - np.pi
    hi_lat = np.pi / 2 - row / Hs * np.pi; lo_lat = np.pi / 2 - (row + 1) / Hs * np.pi
    eps = 1e-12
    assert ((lon >= lo_lon - eps) & (lon <= hi_lon + eps)).all()
    assert ((lat >= lo_lat - eps) & (lat <= hi_lat + eps)).all()
