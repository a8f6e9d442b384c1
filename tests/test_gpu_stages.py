"""Per-stage parity of the CUDA kernels (through the C ABI) against the FP64 oracle.

Sizes span several 32x32 tiles with ragged tails; tolerances are those of the
filter's contract: 1e-4 px/frame max-abs for flows, 1e-5 for inverse depth
and brightness.
"""
import numpy as np
import pytest

import oracle
from paper_2406_18031_b300 import scenes, sf
from tests import gpu_util as gu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    oracle.build()
    oracle.set_threads(8)


def _t(a):
    return torch.from_numpy(gu.f32(a)).cuda()


# ------------------------------------------------------------------ propagation

# 200 x 184 has regions clear of the image border on every side (the
# kernel's interior copy); the others are border regions only
@pytest.mark.parametrize("H,W", [(80, 72), (33, 47), (8, 8), (200, 184)])
@pytest.mark.parametrize("N", [1, 3, 8, 12, 20])
@pytest.mark.parametrize("top", [True, False])
@pytest.mark.parametrize("flags", [0, oracle.SOURCE_SPLIT])
def test_propagate_matches_oracle(H, W, N, top, flags):
    rng = np.random.default_rng(100 + H + N + 7 * top)
    fx = fy = W / 2.0 + 3.0
    cx, cy = W / 2.0 - 1.5, H / 2.0 + 0.5
    g, eta, B, dmu = gu.level_grid(H, W, fx, fy, cx, cy, 1)
    # pixel speeds up to 0.8 N (Eq. 67 holds) but at most a tenth of the grid per
    # frame: on tiny wide-angle grids larger flows are O(1) rad/frame and the
    # source term -w<eta,w> blows the exact solution up
    w = gu.cfl_scaled(gu.flow_field(rng, H, W, dmu, max_px=1.0), eta, B, dmu, min(0.8 * N, 0.1 * min(H, W)))
    rho = gu.f32(0.2 + 0.15 * gu.smooth_field(rng, H, W))
    dw = None if top else gu.f32(gu.flow_field(rng, H, W, dmu, max_px=0.3 * N) * 0.5)
    Y = None if top else gu.f32(0.5 + 0.4 * gu.smooth_field(rng, H, W, n_waves=6))
    s0 = np.concatenate([w, rho[..., None]], -1)
    s1 = None if top else np.concatenate([dw, Y[..., None]], -1)
    o0 = torch.empty((H, W, 4), device="cuda")
    o1 = None if top else torch.empty((H, W, 4), device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    sf.propagate(g, N, _t(s0), o0, None if top else _t(s1), o1, flags=flags | sf.CHECK_CFL, status=status)
    torch.cuda.synchronize()
    rw, rdw, rr, ry, cfl = oracle.propagate(w, rho, eta, B, dmu, N, dw=dw, Y=Y, flags=flags)
    out0 = o0.cpu().numpy()
    assert gu.px_err(out0[..., :3], rw, dmu) <= gu.FLOW_TOL_PX
    assert np.abs(out0[..., 3] - rr).max() <= gu.RHO_TOL
    if not top:
        out1 = o1.cpu().numpy()
        assert gu.px_err(out1[..., :3], rdw, dmu) <= gu.FLOW_TOL_PX
        assert np.abs(out1[..., 3] - ry).max() <= gu.Y_TOL
    # the device flags Eq. 67 exactly when the oracle's CFL number exceeds 1
    # (cases within 1e-5 of the bound may round either way)
    if abs(cfl - 1.0) > 1e-5:
        assert bool(int(status.item()) & 1) == (cfl > 1.0), cfl


@pytest.mark.parametrize("H,W", [(80, 72), (33, 47), (200, 184)])
@pytest.mark.parametrize("N", [1, 3, 12])
@pytest.mark.parametrize("top", [True, False])
@pytest.mark.parametrize("flags", [0, oracle.DOMINANT_LITERAL | oracle.SOURCE_SPLIT])
def test_propagate_inertial_terms_match_oracle(H, W, N, top, flags):
    # SF_IMU: the source step -2 Om x w - Om x (Om x eta) - rho a after each
    # sub-iteration (and -2 Om x dw below the top), Om and a in frame units
    rng = np.random.default_rng(300 + H + N + 7 * top)
    fx = fy = W / 2.0 + 3.0
    g, eta, B, dmu = gu.level_grid(H, W, fx, fy, W / 2.0 - 1.5, H / 2.0 + 0.5, 1)
    w = gu.cfl_scaled(gu.flow_field(rng, H, W, dmu, max_px=1.0), eta, B, dmu, min(0.6 * N, 0.1 * min(H, W)))
    rho = gu.f32(0.2 + 0.15 * gu.smooth_field(rng, H, W))
    dw = None if top else gu.f32(gu.flow_field(rng, H, W, dmu, max_px=0.3 * N) * 0.5)
    Y = None if top else gu.f32(0.5 + 0.4 * gu.smooth_field(rng, H, W, n_waves=6))
    d = float(dmu.mean())
    om = rng.normal(size=3); om *= 0.4 * d / np.linalg.norm(om)          # ~0.4 px/frame of rotation
    ac = rng.normal(size=3); ac *= 0.3 * d / np.linalg.norm(ac) / 0.35   # rho a ~ 0.3 px/frame
    imu = gu.f32(np.concatenate([om, ac]))
    s0 = np.concatenate([w, rho[..., None]], -1)
    s1 = None if top else np.concatenate([dw, Y[..., None]], -1)
    o0 = torch.empty((H, W, 4), device="cuda")
    o1 = None if top else torch.empty((H, W, 4), device="cuda")
    sf.propagate_imu(g, N, imu, _t(s0), o0, None if top else _t(s1), o1, flags=flags)
    torch.cuda.synchronize()
    rw, rdw, rr, ry, _ = oracle.propagate(w, rho, eta, B, dmu, N, dw=dw, Y=Y, flags=oracle.IMU | flags,
                                          imu=imu.astype(np.float64))
    out0 = o0.cpu().numpy()
    assert gu.px_err(out0[..., :3], rw, dmu) <= gu.FLOW_TOL_PX
    assert np.abs(out0[..., 3] - rr).max() <= gu.RHO_TOL
    if not top:
        out1 = o1.cpu().numpy()
        assert gu.px_err(out1[..., :3], rdw, dmu) <= gu.FLOW_TOL_PX
        assert np.abs(out1[..., 3] - ry).max() <= gu.Y_TOL
    # and the terms matter at this size: without them the flow differs
    rw0 = oracle.propagate(w, rho, eta, B, dmu, N, dw=dw, Y=Y, flags=flags)[0]
    assert gu.px_err(out0[..., :3], rw0, dmu) > 100 * gu.FLOW_TOL_PX


def test_propagate_flags_cfl_violation():
    H = W = 40
    g, eta, B, dmu = gu.level_grid(H, W, 20.0, 20.0, 20.0, 20.0, 1)
    w = np.zeros((H, W, 3), np.float32)
    w[..., 0] = 3.0 * dmu     # 3 px/frame with N = 2: dt * |u| = 1.5
    s0 = np.concatenate([w, np.full((H, W, 1), 0.5, np.float32)], -1)
    out = torch.empty((H, W, 4), device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    sf.propagate(g, 2, _t(s0), out, flags=sf.CHECK_CFL, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) & 1
    status.zero_()
    sf.propagate(g, 4, _t(s0), out, flags=sf.CHECK_CFL, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0


def test_propagate_dominant_literal_flag():
    rng = np.random.default_rng(5)
    H, W, N = 64, 40, 4
    g, eta, B, dmu = gu.level_grid(H, W, 30.0, 30.0, 20.0, 32.0, 1)
    w = gu.flow_field(rng, H, W, dmu, 3.0)
    rho = gu.f32(np.full((H, W), 0.3))
    out = torch.empty((H, W, 4), device="cuda")
    sf.propagate(g, N, _t(np.concatenate([w, rho[..., None]], -1)), out, flags=sf.DOMINANT_LITERAL)
    torch.cuda.synchronize()
    rw, _, rr, _, _ = oracle.propagate(w, rho, eta, B, dmu, N, flags=oracle.DOMINANT_LITERAL)
    assert gu.px_err(out.cpu().numpy()[..., :3], rw, dmu) <= gu.FLOW_TOL_PX


# ------------------------------------------------------------------ update

def _update_case(level, levels, top, S, init, seed=11, H1=128, W1=96, invalid=True):
    rng = np.random.default_rng(seed)
    seq = scenes.scene512(frames=2, H=H1, W=W1, seed=seed, max_flow=4.0, levels=levels, iters=[2] * levels,
                          smooth=[2] * levels)
    image, rng_ = seq.image[1].copy(), seq.range[1].copy()
    if invalid:
        image[5:9, 10:30] = 0.9
        rng_[5:9, 10:30] = np.inf          # sky: no measurement
        rng_[40, 40:44] = 0.0
        rng_[50:53, 7] = np.nan
    g, eta, B, dmu = gu.level_grid(H1, W1, seq.fx, seq.fy, seq.cx, seq.cy, level)
    H, W = g.H, g.W
    gam = [1.0, 1.0, 1e-2 * (2 ** (level - 1) / seq.fx) ** 2, 1.0, 1.0]
    s0c = np.concatenate([gu.flow_field(rng, H, W, dmu, 3.0), gu.f32(0.2 + 0.1 * gu.smooth_field(rng, H, W))[..., None]], -1)
    s1c = np.concatenate([gu.flow_field(rng, H, W, dmu, 1.0) * 0, gu.f32(0.5 + 0.3 * gu.smooth_field(rng, H, W))[..., None]], -1)
    p0 = np.concatenate([gu.flow_field(rng, H, W, dmu, 3.0), gu.f32(0.2 + 0.1 * gu.smooth_field(rng, H, W))[..., None]], -1)
    p1 = np.concatenate([gu.flow_field(rng, H, W, dmu, 1.0), gu.f32(0.5 + 0.3 * gu.smooth_field(rng, H, W))[..., None]], -1)
    s0c, s1c, p0, p1 = map(gu.f32, (s0c, s1c, p0, p1))
    n0 = torch.full((H, W, 4), -7.0, device="cuda")
    n1 = torch.full((H, W, 4), -7.0, device="cuda")
    diag = torch.zeros((H, W, 12), device="cuda")
    sf.update(g, level, top, S, init, gam, 1.0, _t(image), _t(rng_), n0, n1, s0_cur=_t(s0c), s1_cur=_t(s1c),
              p0=_t(p0), p1=_t(p1), diag=diag)
    torch.cuda.synchronize()
    Yh, rh, vh = gu.oracle_level_data(image, rng_, level)[level - 1]
    Yhat, _, gY = oracle.image_model(Yh, B, dmu)
    _, gR = oracle.invdepth_model(rh, vh, B, dmu)
    ref = dict(Yhat=Yhat, gY=gY, rh=rh, vh=vh, gR=gR, dmu=dmu)
    if not init:
        if top:
            x = oracle.update(gam[:3], eta, dmu, Yhat, gY, rh, gR, vh, s1c[..., 3], s0c[..., 3], p0[..., :3])
        else:
            x = oracle.update(gam[:3], eta, dmu, Yhat, gY, rh, gR, vh, p1[..., 3], p0[..., 3], p1[..., :3])
        ref["x"] = x
        ref["xs"] = oracle.smooth(x, S)
        ref["rho"] = oracle.blend(gam[3], gam[4], rh, vh, p0[..., 3])
    return ref, n0.cpu().numpy(), n1.cpu().numpy(), diag.cpu().numpy()


@pytest.mark.parametrize("level,levels", [(1, 1), (1, 2), (2, 2), (1, 3), (2, 3), (3, 3), (1, 4), (3, 4), (4, 4)])
@pytest.mark.parametrize("S", [0, 1, 2, 3, 4, 16])   # 2 and 4 take constant strides; 16 the largest region
def test_update_matches_oracle(level, levels, S):
    top = level == levels
    ref, n0, n1, diag = _update_case(level, levels, top, S, init=False)
    dmu = ref["dmu"]
    # measurement models
    assert np.abs(diag[..., 0] - ref["Yhat"]).max() <= 1e-6
    assert gu.px_err(diag[..., 1:4], ref["gY"], dmu) <= 1e-5
    assert np.abs(diag[..., 4] - ref["rh"]).max() <= 1e-6 * max(1.0, np.abs(ref["rh"]).max())
    assert gu.px_err(diag[..., 5:8], ref["gR"], dmu) <= 1e-6
    # solve before smoothing, then the smoothed state
    assert gu.px_err(diag[..., 8:11], ref["x"], dmu) <= gu.FLOW_TOL_PX
    sol = n0[..., :3] if top else n1[..., :3]
    assert gu.px_err(sol, ref["xs"], dmu) <= gu.FLOW_TOL_PX
    assert np.abs(n0[..., 3] - ref["rho"]).max() <= gu.RHO_TOL
    assert np.abs(n1[..., 3] - ref["Yhat"]).max() <= 1e-6
    if top:
        assert (n1[..., :3] == 0).all()


@pytest.mark.parametrize("level,levels", [(1, 1), (2, 2), (3, 3), (1, 3), (4, 4)])
def test_update_init_frame(level, levels):
    ref, n0, n1, _ = _update_case(level, levels, level == levels, 4, init=True)
    assert (n0[..., :3] == 0).all() and (n1[..., :3] == 0).all()
    expect = np.where(ref["vh"] > 0, ref["rh"], 0.0)
    assert np.abs(n0[..., 3] - expect).max() <= 1e-6
    assert np.abs(n1[..., 3] - ref["Yhat"]).max() <= 1e-6


# ------------------------------------------------------------------ reconstruction

@pytest.mark.parametrize("levels", [1, 2, 3, 4])
def test_reconstruct_matches_oracle(levels):
    rng = np.random.default_rng(21 + levels)
    H1, W1 = 96, 136
    grids, s0, s1, ref_w, dmus = [], [], [], [], []
    for h in range(levels):
        g, eta, B, dmu = gu.level_grid(H1, W1, 70.0, 70.0, 68.0, 48.0, h + 1)
        grids.append(g); dmus.append(dmu)
        a = np.concatenate([gu.flow_field(rng, g.H, g.W, dmu, 2.0), gu.f32(rng.uniform(0.1, 0.5, (g.H, g.W, 1)))], -1)
        b = np.concatenate([gu.flow_field(rng, g.H, g.W, dmu, 0.5), gu.f32(rng.uniform(0, 1, (g.H, g.W, 1)))], -1)
        s0.append(_t(a)); s1.append(_t(b))
        ref_w.append((a[..., :3].astype(np.float64), b[..., :3].astype(np.float64), a[..., 3].astype(np.float64)))
    flow = torch.empty((3, H1, W1), device="cuda")
    inv = torch.empty((H1, W1), device="cuda")
    dt = 1 / 600.0
    sf.reconstruct(grids, s0, s1, dt, flow, inv)
    torch.cuda.synchronize()
    w = ref_w[-1][0]
    for h in range(levels - 2, -1, -1):
        w = oracle.upsample_add(w, ref_w[h][1])
        got = s0[h].cpu().numpy()
        assert gu.px_err(got[..., :3], w, dmus[h]) <= 1e-5
    out = np.moveaxis(flow.cpu().numpy(), 0, -1) * dt
    assert gu.px_err(out, w, dmus[0]) <= 1e-5
    assert np.abs(inv.cpu().numpy() - ref_w[0][2]).max() == 0.0
