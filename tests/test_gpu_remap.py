"""Parity of the remapping kernels (sf_remap_pinhole, sf_remap_equirect) with
the oracle, at small and at full sizes (the camera frame 1440 x 720 onto a
1024 x 1024 grid, a 2048 x 1024 panorama onto 512 x 512).

Brightness: within 2e-3 source pixels times the image's largest gradient (FP32
rounding of the projected coordinate, up to a few ulp of a coordinate below
4096).  Range (nearest pixel) and the out-of-view decision are integer
decisions taken from a float coordinate: where the oracle's coordinate is
within 1e-3 px of a pixel edge or of the frame edge, either neighbour (or no
measurement) is accepted; everywhere else the values must be identical."""
import numpy as np
import pytest

import oracle
from paper_2406_18031_b300 import sf
from tests import gpu_util as gu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    oracle.build()
    oracle.set_threads(8)


def _R(ax, ay, az):
    cx, sx, cy, sy, cz, sz = np.cos(ax), np.sin(ax), np.cos(ay), np.sin(ay), np.cos(az), np.sin(az)
    Rx = np.array([[1, 0, 0], [0, cx, -sx], [0, sx, cx]])
    Ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
    Rz = np.array([[cz, -sz, 0], [sz, cz, 0], [0, 0, 1]])
    return gu.f32(Rz @ Ry @ Rx).astype(np.float64)


def _smooth_image(rng, H, W):
    img = 0.5 + 0.4 * gu.smooth_field(rng, H, W, n_waves=6)
    return gu.f32(img)


def _blocky_range(rng, H, W):
    # piecewise constant ranges (occlusion-like edges) in 1..20 m
    lam = np.full((H, W), 15.0)
    for _ in range(12):
        i0, j0 = rng.integers(0, H), rng.integers(0, W)
        lam[i0:i0 + rng.integers(4, H // 2), j0:j0 + rng.integers(4, W // 2)] = rng.uniform(1, 20)
    return gu.f32(lam)


def _max_grad(img, wrap=False):
    gx = np.abs(np.diff(img, axis=1, append=img[:, :1] if wrap else img[:, -1:]))
    gy = np.abs(np.diff(img, axis=0, append=img[-1:]))
    return float(max(gx.max(), gy.max()))


def _grid_rays(g, R):
    j = (np.arange(g.W) + 0.5 - g.cx) / g.fx
    i = (np.arange(g.H) + 0.5 - g.cy) / g.fy
    x, y = np.meshgrid(j, i)
    return np.stack([x, y, np.ones_like(x)], -1) @ np.asarray(R).T


def _check(out_img, out_rng, ref_img, ref_rng, src_img, src_rng, u, v, Hs, Ws, wrap):
    tol = 2e-3 * _max_grad(src_img, wrap) + 1e-6
    edge_u = np.abs(u - np.round(u)) < 1e-3
    edge_v = np.abs(v - np.round(v)) < 1e-3
    frame_edge = np.zeros_like(edge_u) if wrap else (
        (np.abs(u) < 1e-3) | (np.abs(u - Ws) < 1e-3) | (np.abs(v) < 1e-3) | (np.abs(v - Hs) < 1e-3))
    exact = ~(edge_u | edge_v | frame_edge)
    assert np.abs(out_img - ref_img)[~frame_edge].max() <= tol
    assert (out_rng[exact] == ref_rng[exact]).all()
    # the rest: one of the neighbouring source pixels, or no measurement
    for i, j in zip(*np.nonzero(~exact)):
        jn, in_ = int(np.floor(u[i, j])), int(np.floor(v[i, j]))
        cand = {0.0}
        for di in (-1, 0, 1):
            for dj in (-1, 0, 1):
                ii = min(max(in_ + di, 0), Hs - 1)
                jj = (jn + dj) % Ws if wrap else min(max(jn + dj, 0), Ws - 1)
                cand.add(float(src_rng[ii, jj]))
        assert float(out_rng[i, j]) in cand


def _pinhole_case(Hs, Ws, cam, g, R, seed):
    rng = np.random.default_rng(seed)
    img, lam = _smooth_image(rng, Hs, Ws), _blocky_range(rng, Hs, Ws)
    oi = torch.empty((g.H, g.W), device="cuda"); orng = torch.empty((g.H, g.W), device="cuda")
    sf.remap_pinhole(g, R, cam, torch.from_numpy(img).cuda(), oi, torch.from_numpy(lam).cuda(), orng)
    torch.cuda.synchronize()
    ri, rr = oracle.remap_pinhole(g.H, g.W, (g.fx, g.fy, g.cx, g.cy), R, cam, img, lam)
    d = _grid_rays(g, R)
    with np.errstate(divide="ignore", invalid="ignore"):
        u = np.where(d[..., 2] > 0, cam[0] * d[..., 0] / d[..., 2] + cam[2], -1e9)
        v = np.where(d[..., 2] > 0, cam[1] * d[..., 1] / d[..., 2] + cam[3], -1e9)
    _check(oi.cpu().numpy(), orng.cpu().numpy(), ri, rr, img, lam, u, v, Hs, Ws, False)
    return ri, rr


@pytest.mark.parametrize("R", [(0.0, 0.0, 0.0), (0.05, -0.3, 0.2), (0.0, 0.9, 0.0)], ids=["ident", "tilted", "sideways"])
def test_pinhole_small(R):
    g = sf.grid(96, 128, 60.0, 60.0, 64.0, 48.0)
    ri, rr = _pinhole_case(90, 180, (88.0, 86.0, 91.5, 44.0), g, _R(*R), seed=7)
    assert (rr > 0).any()


def test_pinhole_full_size_camera_frame_onto_1024_grid():
    # a 1440 x 720 camera (about 110 x 70 degrees) onto a 1024 x 1024 grid of
    # about the same horizontal field of view, slightly rotated
    g = sf.grid(1024, 1024, 360.0, 360.0, 512.0, 512.0)
    _pinhole_case(720, 1440, (500.0, 500.0, 720.0, 360.0), g, _R(0.02, 0.05, -0.01), seed=8)


def _equirect_case(Hs, g, R, seed):
    Ws = 2 * Hs
    rng = np.random.default_rng(seed)
    img, lam = _smooth_image(rng, Hs, Ws), _blocky_range(rng, Hs, Ws)
    oi = torch.empty((g.H, g.W), device="cuda"); orng = torch.empty((g.H, g.W), device="cuda")
    sf.remap_equirect(g, R, torch.from_numpy(img).cuda(), oi, torch.from_numpy(lam).cuda(), orng)
    torch.cuda.synchronize()
    ri, rr = oracle.remap_equirect(g.H, g.W, (g.fx, g.fy, g.cx, g.cy), R, img, lam)
    d = _grid_rays(g, R)
    d = d / np.linalg.norm(d, axis=-1, keepdims=True)
    u = (np.arctan2(d[..., 0], d[..., 2]) + np.pi) / (2 * np.pi) * Ws
    v = (np.pi / 2 - np.arcsin(-d[..., 1])) / np.pi * Hs
    _check(oi.cpu().numpy(), orng.cpu().numpy(), ri, rr, img, lam, u, v, Hs, Ws, True)


@pytest.mark.parametrize("R", [(0.0, 0.0, 0.0), (0.4, 3.1, 0.1)], ids=["forward", "across_the_wrap"])
def test_equirect_small(R):
    _equirect_case(128, sf.grid(80, 96, 40.0, 40.0, 48.0, 40.0), _R(*R), seed=9)


def test_equirect_full_size_panorama_onto_512_grid():
    # the paper's rendering path: a 360-degree panorama onto a front-facing
    # 512 x 512 grid (90 degree field of view)
    _equirect_case(1024, sf.grid(512, 512, 256.0, 256.0, 256.0, 256.0), _R(0.0, 0.0, 0.0), seed=10)


def test_binding_rejects_wrong_buffers_before_the_call():
    g = sf.CGrid(16, 24, 20.0, 20.0, 11.5, 7.5)
    R = np.eye(3)
    img = torch.zeros((10, 12), device="cuda")
    oi = torch.empty((16, 24), device="cuda")
    with pytest.raises(ValueError, match="out_image: expected 384"):
        sf.remap_pinhole(g, R, (10.0, 10.0, 6.0, 5.0), img, oi[:, :-1])
    with pytest.raises(ValueError, match="rng: expected 120"):
        sf.remap_pinhole(g, R, (10.0, 10.0, 6.0, 5.0), img, oi, torch.zeros((10, 11), device="cuda"), oi.clone())
    with pytest.raises(ValueError, match="image: expected"):
        sf.remap_equirect(g, R, img.double(), oi)
    with pytest.raises(ValueError, match="out_range: expected 384"):
        sf.remap_equirect(g, R, img, oi, img.clone(), torch.empty(383, device="cuda"))
    sf.remap_equirect(g, R, img, oi)                                   # the right ones still work
    torch.cuda.synchronize()
    assert float(oi.abs().max()) == 0.0
