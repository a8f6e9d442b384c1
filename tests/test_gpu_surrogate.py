"""The learned propagation surrogate on the GPU against the oracle's float64
statement of the same network (oracle/surrogate.py), which rounds to
bfloat16 at the points where the CUDA path stores bfloat16.

Forward: the prediction agrees within 2^-7 of the largest output (one
bfloat16 ulp of a value that may round differently when its float32 and
float64 sums straddle a rounding boundary) plus 1e-4 (float32 accumulation),
in the network's units.  Gradients: every weight and bias within (2^-7 +
n 2^-23) of the |.|-weighted sum of the products that form it
(tests/surrogate_bounds.py: one bfloat16 ulp for the isolated stores and ReLU
decisions that round differently, float32 accumulation over n pixels).
Training: 400 Adam steps on pairs
produced by the plain propagation lower the loss at least five-fold."""
import numpy as np
import pytest

import oracle
from oracle import surrogate as S
from paper_2406_18031_b300 import sf
from tests import gpu_util as gu
from tests import surrogate_bounds as SB

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    oracle.build()


def _states(rng, n, H, W, dmu, eta, B, max_px):
    out = []
    for _ in range(n):
        w = gu.cfl_scaled(gu.flow_field(rng, H, W, dmu, max_px=1.0), eta, B, dmu, max_px)
        rho = gu.f32(0.2 + 0.15 * gu.smooth_field(rng, H, W))
        out.append(np.concatenate([w, rho[..., None]], -1))
    return gu.f32(np.stack(out))


def _layer_slices():
    k, out = 0, []
    for cin, cout in S.LAYERS:
        out.append(slice(k, k + 9 * cin * cout + cout))
        k += 9 * cin * cout + cout
    return out


# the fused kernel (k_surr_net: tiles of 120 columns, strips of 16..64 rows)
# and the layered form; 40 x 160: two tiles, the second ragged; 33 x 47: one
# ragged tile shorter than a strip; 130 x 250, one frame: strips of 16 rows,
# three tiles
@pytest.mark.parametrize("form", ["fused", "layered"])
@pytest.mark.parametrize("n,H,W", [(2, 40, 160), (3, 33, 47), (1, 130, 250)])
def test_forward_matches_oracle(form, n, H, W):
    rng = np.random.default_rng(1 + H)
    g, eta, B, dmu = gu.level_grid(H, W, 0.5 * W, 0.5 * W, 0.5 * W, 0.5 * H, 1)
    net = sf.Surrogate(seed=3)
    p = net.params()
    p[-16 - 9 * 16 * 32:] *= 10.0          # a larger last layer than at creation: visible outputs
    net.set_params(p)
    s0 = _states(rng, n, H, W, dmu, eta, B, 1.5)
    p0 = torch.full(s0.shape, np.nan, device="cuda")
    net.forward(g, torch.from_numpy(s0).cuda(), p0, layered=form == "layered")
    torch.cuda.synchronize()
    _, y = S.forward(S.features(eta, dmu, s0), p, q=S.bf16)
    ref = np.empty_like(s0, dtype=np.float64)
    ref[..., 0:3] = s0[..., 0:3] + 4 * dmu[None, ..., None] * y[..., 0:3]
    ref[..., 3] = s0[..., 3] + y[..., 3]
    got = p0.cpu().numpy().astype(np.float64)
    tol = 2.0 ** -7 * np.abs(y[..., :4]).max() + 1e-4
    assert np.abs((got[..., 0:3] - ref[..., 0:3]) / (4 * dmu[None, ..., None])).max() <= tol
    assert np.abs(got[..., 3] - ref[..., 3]).max() <= tol


# (4, 1024, 1024) runs strips of 256 rows, (1, 1024, 1024) of 64, (2, 96, 312) of 16;
# 65 frames take two launches (64 images at most per launch)
@pytest.mark.parametrize("n,H,W", [(4, 1024, 1024), (1, 1024, 1024), (2, 96, 312), (1, 8, 8), (65, 16, 24)])
def test_fused_forward_matches_layered(n, H, W):
    # the same arithmetic at the same rounding points: the tensor cores' sums
    # in the same order, bias and ReLU in float32, bfloat16 stores of the
    # hidden activations (in shared memory instead of HBM), the same head
    rng = np.random.default_rng(7 + W)
    g, eta, B, dmu = gu.level_grid(H, W, 0.5 * W, 0.5 * W, 0.5 * W, 0.5 * H, 1)
    net = sf.Surrogate(seed=5)
    p = net.params()
    p[-16 - 9 * 16 * 32:] *= 10.0
    net.set_params(p)
    s0 = torch.from_numpy(_states(rng, n, H, W, dmu, eta, B, 2.0)).cuda()
    a = torch.full(s0.shape, np.nan, device="cuda")
    b = torch.full(s0.shape, np.nan, device="cuda")
    for _ in range(2):                      # twice: the second call reuses the buffers
        net.forward(g, s0, a)
        net.forward(g, s0, b, layered=True)
    torch.cuda.synchronize()
    assert torch.isfinite(a).all()
    d = (a - b).abs().max().item()
    scale = (b - s0).abs().max().item()
    assert scale > 0
    assert d <= 1e-6 * scale, (d, scale)


def test_fused_network_bounded_waits_give_up_and_leave_the_device_usable():
    # a frame whose MMAs are never issued: the fused kernel's waits cannot
    # succeed; it must report the timeout, free its tensor memory and return
    assert sf.lib().sf_selftest_net_timeout(None) == sf.ETIMEOUT
    rng = np.random.default_rng(3)
    g, eta, B, dmu = gu.level_grid(16, 40, 20.0, 20.0, 20.0, 8.0, 1)
    net = sf.Surrogate(seed=5)
    s0 = torch.from_numpy(_states(rng, 1, 16, 40, dmu, eta, B, 1.0)).cuda()
    a, b = torch.empty_like(s0), torch.empty_like(s0)
    net.forward(g, s0, a)                   # and the next forward still works
    net.forward(g, s0, b, layered=True)
    torch.cuda.synchronize()
    assert torch.isfinite(a).all()
    assert (a - b).abs().max().item() <= 1e-6 * max((b - s0).abs().max().item(), 1e-6)


def test_gradients_match_oracle():
    rng = np.random.default_rng(2)
    H, W = 24, 136
    g, eta, B, dmu = gu.level_grid(H, W, 70.0, 70.0, 68.0, 12.0, 1)
    net = sf.Surrogate(seed=5)
    p = net.params()
    p[-16 - 9 * 16 * 32:] *= 10.0
    net.set_params(p)
    s0 = _states(rng, 2, H, W, dmu, eta, B, 1.0)
    tgt = gu.f32(s0 + rng.normal(size=s0.shape) * np.concatenate([np.broadcast_to(dmu[..., None], (H, W, 3)) * 0.3,
                                                                    np.full((H, W, 1), 0.01)], -1)[None])
    loss = net.train_step(g, torch.from_numpy(s0).cuda(), torch.from_numpy(tgt).cuda(), lr=0.0)
    gg = net.grads()
    ref_loss, ref_g, tol = SB.oracle_gradients_and_tolerance(S.features(eta, dmu, s0), p,
                                                             S.residual_target(eta, dmu, s0, tgt))
    assert abs(loss - ref_loss) <= 1e-3 * ref_loss
    # element by element: every weight and bias of every layer
    bad = np.abs(gg - ref_g) > tol
    assert not bad.any(), (int(bad.sum()), np.flatnonzero(bad)[:8], (np.abs(gg - ref_g) / np.maximum(tol, 1e-300)).max())
    # the comparison is not vacuous: the gradients are far from zero and the
    # tolerance is a small fraction of them
    for sl in _layer_slices():
        nz = ref_g[sl] != 0
        assert nz.mean() > 0.2 and np.median(tol[sl][nz] / np.abs(ref_g[sl][nz])) < 0.05
    np.testing.assert_array_equal(net.params(), p)     # lr = 0 leaves the parameters


def test_training_on_plain_propagation_pairs_lowers_the_loss():
    rng = np.random.default_rng(3)
    H, W, N = 64, 256, 2
    g, eta, B, dmu = gu.level_grid(H, W, 128.0, 128.0, 128.0, 32.0, 1)
    s0 = _states(rng, 8, H, W, dmu, eta, B, 1.5)
    s0_t = torch.from_numpy(s0).cuda()
    tgt = torch.empty_like(s0_t)
    for k in range(s0.shape[0]):
        sf.propagate(g, N, s0_t[k], tgt[k])
    net = sf.Surrogate(seed=7)
    losses = [net.train_step(g, s0_t, tgt, lr=2e-3) for _ in range(400)]
    assert np.isfinite(losses).all()
    assert min(losses[-20:]) < 0.2 * losses[0], (losses[0], losses[-1])


def test_fallback_to_the_plain_propagation():
    rng = np.random.default_rng(4)
    H, W, N = 32, 192, 3
    g, eta, B, dmu = gu.level_grid(H, W, 96.0, 96.0, 96.0, 16.0, 1)
    s0 = torch.from_numpy(_states(rng, 2, H, W, dmu, eta, B, 1.0)).cuda()
    net = sf.Surrogate(seed=9)
    fwd = torch.empty_like(s0); net.forward(g, s0, fwd)
    plain = torch.empty_like(s0)
    for k in range(2):
        sf.propagate(g, N, s0[k], plain[k])
    out = torch.empty_like(s0)
    res, used = net.propagate(g, N, s0, out, threshold_px=1e30)
    torch.cuda.synchronize()
    assert not used and res > 0
    assert torch.equal(out, fwd)
    res2, used2 = net.propagate(g, N, s0, out, threshold_px=0.5 * res)
    torch.cuda.synchronize()
    assert used2 and abs(res2 - res) <= 1e-6 * res
    assert torch.equal(out, plain)


def _planar_to_state(planes):
    """[8, H, W] checkpoint planes -> (s0, s1) as [H, W, 4] float32 tensors."""
    return planes[0:4].permute(1, 2, 0).contiguous(), planes[4:8].permute(1, 2, 0).contiguous()


def test_filter_top_level_predicted_by_the_surrogate():
    # a single-level filter with the surrogate attached computes, per frame,
    # the surrogate's prediction of its state followed by the update: the same
    # as the stage entry points chained by hand
    from paper_2406_18031_b300 import scenes
    seq = scenes.plane64(frames=3, H=48, W=160, levels=1, iters=[2])
    H, W = seq.shape
    P = sf.Params(fx=seq.fx, fy=seq.fy, cx=seq.cx, cy=seq.cy, iters=seq.iters, smooth=seq.smooth)
    net = sf.Surrogate(seed=11)
    p = net.params(); p[-16 - 9 * 16 * 32:] *= 10.0; net.set_params(p)
    filt = sf.Filter(H, W, 1, P)
    filt.set_surrogate(net)
    filt.set_surrogate_threshold(float("inf"))            # the prediction is always accepted here
    img = [torch.from_numpy(seq.image[k]).cuda() for k in range(3)]
    rng_ = [torch.from_numpy(seq.range[k]).cuda() for k in range(3)]
    flow = torch.empty((3, H, W), device="cuda")
    filt.step(img[0], rng_[0], seq.dt, flow)
    planes, _ = filt.get_state(0)
    s0, s1 = _planar_to_state(planes)
    filt.step(img[1], rng_[1], seq.dt, flow)
    got, _ = filt.get_state(0)
    g = sf.grid(H, W, seq.fx, seq.fy, seq.cx, seq.cy)
    p0 = torch.empty_like(s0)
    net.forward(g, s0[None], p0[None])
    gam = list(filt.params.gamma)
    gam[2] = gam[2] / seq.fx ** 2                         # the level-1 prior weight (reading R10)
    n0, n1 = torch.empty_like(s0), torch.empty_like(s0)
    sf.update(g, 1, 1, seq.smooth[0], 0, gam, 1.0, img[1], rng_[1], n0, n1, s0, s1, p0, None)
    torch.cuda.synchronize()
    ref = torch.cat([n0.permute(2, 0, 1), n1.permute(2, 0, 1)])
    assert torch.equal(got, ref)
    # the fused surrogate (features and network in one launch), the fallback check
    # (one plain step reduced to the residual, the gated plain propagation), solve,
    # smoothing
    assert filt.kernels_per_step() == 1 + 2 + 1 + 1
    res, fell = filt.surrogate_stats()
    assert res > 0 and fell == 0
    # the residual is the stand-alone check's: the largest flow difference of the
    # surrogate's prediction to one plain step, in px/frame
    out = torch.empty_like(s0)
    res_ref, used = net.propagate(g, seq.iters[0], s0[None], out[None], threshold_px=float("inf"))
    torch.cuda.synchronize()
    # (the engine's check takes dmu from the propagation's fast per-pixel geometry:
    # a few ulp from the stand-alone reduction's)
    assert not used and abs(res - res_ref) <= 1e-5 * res_ref, (res, res_ref)


# widths 128 and 192: one fused launch per stream; three streams on one grid:
# one fused launch for all three (separate state planes)
@pytest.mark.parametrize("widths", [(128, 192), (128, 128, 128)])
def test_batch_with_the_surrogate_matches_single_filters(widths):
    from paper_2406_18031_b300 import scenes
    seqs = [scenes.plane64(frames=6, seed=21 + k, H=64, W=w, levels=1, iters=[2]) for k, w in enumerate(widths)]
    net = sf.Surrogate(seed=12)
    P = [sf.Params(fx=q.fx, fy=q.fy, cx=q.cx, cy=q.cy, iters=q.iters, smooth=q.smooth) for q in seqs]
    batch = sf.Batch([q.shape for q in seqs], [1] * len(seqs), P)
    batch.set_surrogate(net)
    singles = [sf.Filter(*q.shape, 1, p) for q, p in zip(seqs, P)]
    net2 = sf.Surrogate(seed=12)            # same weights, its own buffers
    for f in singles:
        f.set_surrogate(net2)
    stream = torch.cuda.Stream()
    outs = [torch.empty((3, *q.shape), device="cuda") for q in seqs]
    dt = seqs[0].dt
    for k in range(6):
        with torch.cuda.stream(stream):
            for s, q in enumerate(seqs):
                batch.slots[s][0].copy_(torch.from_numpy(q.image[k]).cuda())
                batch.slots[s][1].copy_(torch.from_numpy(q.range[k]).cuda())
                singles[s].step(torch.from_numpy(q.image[k]).cuda(), torch.from_numpy(q.range[k]).cuda(), dt,
                                outs[s], stream=stream)
            batch.step(dt, stream=stream)
        stream.synchronize()
        for s in range(len(seqs)):
            assert torch.equal(batch.slots[s][2], outs[s]), (k, s)


def test_batch_fallback_inside_the_captured_step():
    # three single-level streams stepped by three batches through the same
    # frames: P without a surrogate, S with the surrogate always accepted
    # (threshold inf) and A with per-stream thresholds: stream 0 always falls
    # back (threshold 0), stream 1 never (inf), stream 2 on the default
    # threshold.  From the fourth frame on every step replays a captured
    # graph, so the decisions are taken on the device.  A's stream 0 must
    # equal P's bit for bit, its stream 1 S's; stream 2 follows P or S on each
    # frame as its counter says.
    from paper_2406_18031_b300 import scenes
    seqs = [scenes.plane64(frames=8, seed=31 + k, H=64, W=128 + 32 * k, levels=1, iters=[3]) for k in range(3)]
    net = sf.Surrogate(seed=13)
    p = net.params(); p[-16 - 9 * 16 * 32:] *= 10.0; net.set_params(p)
    P = [sf.Params(fx=q.fx, fy=q.fy, cx=q.cx, cy=q.cy, iters=q.iters, smooth=q.smooth) for q in seqs]
    shapes = [q.shape for q in seqs]
    bp, bs, ba = (sf.Batch(shapes, [1] * 3, P) for _ in range(3))
    nets = [sf.Surrogate(seed=13) for _ in range(2)]
    for nn in nets:
        nn.set_params(p)
    bs.set_surrogate(nets[0]); bs.set_surrogate_threshold(float("inf"))
    ba.set_surrogate(nets[1])
    ba.set_surrogate_threshold(0.0, 0); ba.set_surrogate_threshold(float("inf"), 1)
    stream = torch.cuda.Stream()
    dt = seqs[0].dt
    fell_prev = np.zeros(3, np.int64)
    for k in range(8):
        with torch.cuda.stream(stream):
            for b in (bp, bs, ba):
                for s_, q in enumerate(seqs):
                    b.slots[s_][0].copy_(torch.from_numpy(q.image[k]).cuda())
                    b.slots[s_][1].copy_(torch.from_numpy(q.range[k]).cuda())
                b.step(dt, stream=stream)
        stream.synchronize()
        res, fell = ba.surrogate_stats()
        assert torch.equal(ba.slots[0][2], bp.slots[0][2]), k
        assert torch.equal(ba.slots[1][2], bs.slots[1][2]), k
        if k > 0:
            assert fell[0] == k and fell[1] == 0
            assert fell[2] - fell_prev[2] == int(res[2] > 1.0)
        fell_prev = fell
    assert fell_prev[0] == 7
    # the always-accepted batch never ran the fallback
    assert (bs.surrogate_stats()[1] == 0).all()
    for b in (bp, bs, ba):
        b.close()
