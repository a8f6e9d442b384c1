"""Batched streams (sf_batch_*): every stream computes what its own sf_step
computes, through the plain launches and the replayed CUDA graphs."""
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


def _streams():
    return [
        scenes.plane64(frames=7, seed=11, H=64, W=64, levels=1, iters=[2]),
        scenes.plane64(frames=7, seed=12, H=96, W=128, levels=2, iters=[3, 2], v=(2.0, -1.0, 3.0)),
        scenes.scene512(frames=7, seed=13, H=128, W=128, max_flow=3.0, levels=3, iters=(3, 2, 1), smooth=(2, 4, 4)),
        scenes.plane64(frames=7, seed=14, H=64, W=96, levels=2, iters=[10, 5], v=(6.0, 3.0, 1.0)),
    ]


def _params(seq, nf_max=None, update_mode=None):
    return sf.Params(fx=seq.fx, fy=seq.fy, cx=seq.cx, cy=seq.cy, iters=seq.iters, smooth=seq.smooth,
                     flags=sf.CHECK_CFL | sf.CHECK_FINITE, nf_max=nf_max, update_mode=update_mode)


def test_batch_inertial_terms_match_single_stream_filters():
    # SF_IMU: each stream's motion slot, written on the device before the step,
    # against single-stream filters given the same motion by sf_set_motion
    seqs = _streams()[:3]
    dt = seqs[0].dt
    P = [sf.Params(fx=q.fx, fy=q.fy, cx=q.cx, cy=q.cy, iters=q.iters, smooth=q.smooth,
                   flags=sf.CHECK_CFL | sf.CHECK_FINITE | sf.IMU) for q in seqs]
    batch = sf.Batch([q.shape for q in seqs], [q.levels for q in seqs], P)
    singles = [sf.Filter(*q.shape, q.levels, p) for q, p in zip(seqs, P)]
    rng = np.random.default_rng(4)
    stream = torch.cuda.Stream()
    outs = [(torch.empty((3, *q.shape), device="cuda"), torch.empty(q.shape, device="cuda")) for q in seqs]
    for k in range(5):
        with torch.cuda.stream(stream):
            for s, q in enumerate(seqs):
                om, acc = rng.normal(size=3) * 2.0, rng.normal(size=3) * 5.0   # rad/s, m/s^2
                img, rg, _, _ = batch.slots[s]
                img.copy_(torch.from_numpy(q.image[k]).cuda())
                rg.copy_(torch.from_numpy(q.range[k]).cuda())
                batch.motion[s].copy_(torch.tensor(np.concatenate([om, acc]), dtype=torch.float32))
                singles[s].set_motion(om, acc, stream=stream)
                singles[s].step(torch.from_numpy(q.image[k]).cuda(), torch.from_numpy(q.range[k]).cuda(), dt,
                                outs[s][0], outs[s][1], stream=stream)
            batch.step(dt, stream=stream)
        stream.synchronize()
        for s, q in enumerate(seqs):
            _, _, dmu = oracle.geometry(*q.shape, q.fx, q.fy, q.cx, q.cy)
            e = np.abs(batch.slots[s][2].cpu().numpy().astype(np.float64) - outs[s][0].cpu().numpy()) * dt / dmu[None]
            assert e.max() <= gu.FLOW_TOL_PX, (k, s, e.max())
    assert batch.status() in (sf.OK, sf.WARN_CFL)


@pytest.mark.parametrize("nf_max,update_mode", [(None, None), (4, None), (None, 2)])
def test_batch_matches_single_stream_filters_and_oracle(nf_max, update_mode):
    seqs = _streams()
    dt = seqs[0].dt
    assert all(abs(s.dt - dt) < 1e-15 for s in seqs)
    batch = sf.Batch([s.shape for s in seqs], [s.levels for s in seqs],
                     [_params(s, nf_max, update_mode) for s in seqs])
    singles = [sf.Filter(*s.shape, s.levels, _params(s)) for s in seqs]
    ref = oracle.Filter(*seqs[2].shape, seqs[2].levels,
                        oracle.Params(seqs[2].fx, seqs[2].fy, seqs[2].cx, seqs[2].cy, iters=seqs[2].iters,
                                      smooth=seqs[2].smooth))
    _, _, dmu_ref = ref.geometry(0)
    stream = torch.cuda.Stream()
    outs = [(torch.empty((3, *s.shape), device="cuda"), torch.empty(s.shape, device="cuda")) for s in seqs]
    for k in range(7):
        with torch.cuda.stream(stream):
            for s, seq in enumerate(seqs):
                img, rng, _, _ = batch.slots[s]
                img.copy_(torch.from_numpy(seq.image[k]).cuda())
                rng.copy_(torch.from_numpy(seq.range[k]).cuda())
            batch.step(dt, stream=stream)
            for s, seq in enumerate(seqs):
                singles[s].step(torch.from_numpy(seq.image[k]).cuda(), torch.from_numpy(seq.range[k]).cuda(),
                                dt, outs[s][0], outs[s][1], stream=stream)
        stream.synchronize()
        for s, seq in enumerate(seqs):
            _, _, dmu = oracle.geometry(*seq.shape, seq.fx, seq.fy, seq.cx, seq.cy)
            bf, bi = batch.slots[s][2].cpu().numpy(), batch.slots[s][3].cpu().numpy()
            sf_, si = outs[s][0].cpu().numpy(), outs[s][1].cpu().numpy()
            e = np.abs(bf.astype(np.float64) - sf_) * dt / dmu[None]
            assert e.max() <= gu.FLOW_TOL_PX, (k, s, e.max())
            assert np.abs(bi - si).max() <= gu.RHO_TOL
        rf, ri = ref.step(seqs[2].image[k], seqs[2].range[k], dt)
        e = np.abs(batch.slots[2][2].cpu().numpy().astype(np.float64) - rf) * dt / dmu_ref[None]
        assert e.max() <= gu.FLOW_TOL_PX
    # N = 10 on stream 3 needs two propagation launches (three at nf_max = 4),
    # then one solve launch and a smoothing + reconstruction cascade of three
    # levels (update mode 2: one smoothing launch and two reconstruction launches)
    assert batch.launches_per_step() == (2 if nf_max is None else 3) + 1 + 3
    assert batch.update_mode() == (update_mode or 1)
    assert batch.nf_max() == (nf_max or 8)
    assert batch.solve_tile() == 16        # 49 tiles of 32 pixels: one wave
    assert batch.status() in (sf.OK, sf.WARN_CFL)


@pytest.mark.slow
def test_full_size_batch_sampled_streams():
    """The benchmark's batch as it is timed: 64 streams (16 x 256^2 with 2
    levels, 32 x 512^2 and 16 x 1024^2 with 3), the autotuner on, steady-state
    steps replayed from CUDA graphs.  Sampled streams (the first and last of
    each size) against their own single-stream filters every frame, and the
    first 256^2 stream against the FP64 oracle."""
    import bench
    frames = 5
    seqs = scenes.batch(frames=frames, sizes=bench.BATCH_SIZES, period=bench.BATCH_FRAMES)
    assert len(seqs) == 64 and sum(q.shape[0] * q.shape[1] for q in seqs) == 26_214_400
    dt = seqs[0].dt
    flags = sf.CHECK_CFL | sf.CHECK_FINITE | sf.AUTOTUNE
    P = [sf.Params(fx=q.fx, fy=q.fy, cx=q.cx, cy=q.cy, iters=q.iters, smooth=q.smooth, flags=flags) for q in seqs]
    batch = sf.Batch([q.shape for q in seqs], [q.levels for q in seqs], P)
    bounds = np.cumsum([0] + [n for _, n in bench.BATCH_SIZES])
    sample = sorted({int(b) for b in bounds[:-1]} | {int(b) - 1 for b in bounds[1:]})
    singles = {s: sf.Filter(*seqs[s].shape, seqs[s].levels, P[s]) for s in sample}
    q0 = seqs[0]
    ref = oracle.Filter(*q0.shape, q0.levels, oracle.Params(q0.fx, q0.fy, q0.cx, q0.cy, iters=q0.iters,
                                                            smooth=q0.smooth))
    _, _, dmu0 = ref.geometry(0)
    outs = {s: (torch.empty((3, *seqs[s].shape), device="cuda"), torch.empty(seqs[s].shape, device="cuda"))
            for s in sample}
    stream = torch.cuda.Stream()
    for k in range(frames):
        with torch.cuda.stream(stream):
            for s, q in enumerate(seqs):
                img, rng, _, _ = batch.slots[s]
                img.copy_(torch.from_numpy(q.image[k]).cuda())
                rng.copy_(torch.from_numpy(q.range[k]).cuda())
            batch.step(dt, stream=stream)
            for s in sample:
                singles[s].step(torch.from_numpy(seqs[s].image[k]).cuda(), torch.from_numpy(seqs[s].range[k]).cuda(),
                                dt, outs[s][0], outs[s][1], stream=stream)
        stream.synchronize()
        for s in sample:
            q = seqs[s]
            _, _, dmu = oracle.geometry(*q.shape, q.fx, q.fy, q.cx, q.cy)
            e = np.abs(batch.slots[s][2].cpu().numpy().astype(np.float64) - outs[s][0].cpu().numpy()) * dt / dmu[None]
            assert e.max() <= gu.FLOW_TOL_PX, (k, s, e.max())
            assert np.abs(batch.slots[s][3].cpu().numpy() - outs[s][1].cpu().numpy()).max() <= gu.RHO_TOL, (k, s)
        rf, ri = ref.step(q0.image[k], q0.range[k], dt)
        e = np.abs(batch.slots[0][2].cpu().numpy().astype(np.float64) - rf) * dt / dmu0[None]
        assert e.max() <= gu.FLOW_TOL_PX, (k, e.max())
        assert np.abs(batch.slots[0][3].cpu().numpy() - ri).max() <= gu.RHO_TOL, k
    assert batch.status() in (sf.OK, sf.WARN_CFL)


def test_batch_with_a_four_level_stream():
    # streams of 1 to 4 levels in one engine: the deepest sets the number of
    # smoothing depths; each stream against its own single-stream filter
    seqs = [scenes.scene512(frames=4, seed=31, H=128, W=160, max_flow=4.0, levels=4, iters=(4, 2, 1, 1),
                            smooth=(2, 4, 4, 4)),
            scenes.plane64(frames=4, seed=32, H=64, W=64, levels=1, iters=[2])]
    dt = seqs[0].dt
    batch = sf.Batch([q.shape for q in seqs], [q.levels for q in seqs], [_params(q) for q in seqs])
    singles = [sf.Filter(*q.shape, q.levels, _params(q)) for q in seqs]
    outs = [(torch.empty((3, *q.shape), device="cuda"), torch.empty(q.shape, device="cuda")) for q in seqs]
    stream = torch.cuda.Stream()
    for k in range(4):
        with torch.cuda.stream(stream):
            for s, q in enumerate(seqs):
                img, rng, _, _ = batch.slots[s]
                img.copy_(torch.from_numpy(q.image[k]).cuda())
                rng.copy_(torch.from_numpy(q.range[k]).cuda())
            batch.step(dt, stream=stream)
            for s, q in enumerate(seqs):
                singles[s].step(torch.from_numpy(q.image[k]).cuda(), torch.from_numpy(q.range[k]).cuda(), dt,
                                outs[s][0], outs[s][1], stream=stream)
        stream.synchronize()
        for s, q in enumerate(seqs):
            _, _, dmu = oracle.geometry(*q.shape, q.fx, q.fy, q.cx, q.cy)
            e = np.abs(batch.slots[s][2].cpu().numpy().astype(np.float64) - outs[s][0].cpu().numpy()) * dt / dmu[None]
            assert e.max() <= gu.FLOW_TOL_PX, (k, s, e.max())
            assert np.abs(batch.slots[s][3].cpu().numpy() - outs[s][1].cpu().numpy()).max() <= gu.RHO_TOL
    assert batch.status() in (sf.OK, sf.WARN_CFL)


@pytest.mark.slow
def test_list_scheduled_batch_matches_single_stream_filters():
    # A full-size driving stream (384 x 1248, N = [32, 16, 8]) and a full-size
    # 512 x 512 stream (N = [8, 4]) in one batch: the driving levels' segments
    # and the other stream's single segment are list-scheduled together into
    # eight one-wave launches (1,096 tiles), while the single-stream filters
    # run seven (driving) and one (512 x 512) launches.  Every tile computes
    # the same arithmetic on the same inputs in either schedule, so the outputs
    # agree bitwise; the driving stream is also held against the FP64 oracle.
    # One frame time for both (the state is per frame: dt only scales the
    # returned flow), the driving sequence's.
    seqs = [scenes.drive(frames=3), scenes.scene512(frames=3)]
    dt = seqs[0].dt

    def params(seq):
        return sf.Params(fx=seq.fx, fy=seq.fy, cx=seq.cx, cy=seq.cy, iters=seq.iters, smooth=seq.smooth,
                         flags=sf.CHECK_CFL | sf.CHECK_FINITE, nf_max=8, update_mode=1, solve_tile=32)

    batch = sf.Batch([s.shape for s in seqs], [s.levels for s in seqs], [params(s) for s in seqs])
    singles = [sf.Filter(*s.shape, s.levels, params(s)) for s in seqs]
    ref = oracle.Filter(*seqs[0].shape, seqs[0].levels,
                        oracle.Params(seqs[0].fx, seqs[0].fy, seqs[0].cx, seqs[0].cy, iters=seqs[0].iters,
                                      smooth=seqs[0].smooth))
    _, _, dmu_ref = ref.geometry(0)
    stream = torch.cuda.Stream()
    outs = [(torch.empty((3, *s.shape), device="cuda"), torch.empty(s.shape, device="cuda")) for s in seqs]
    for k in range(3):
        with torch.cuda.stream(stream):
            for s, seq in enumerate(seqs):
                img, rng, _, _ = batch.slots[s]
                img.copy_(torch.from_numpy(seq.image[k]).cuda())
                rng.copy_(torch.from_numpy(seq.range[k]).cuda())
                singles[s].step(torch.from_numpy(seq.image[k]).cuda(), torch.from_numpy(seq.range[k]).cuda(),
                                dt, outs[s][0], outs[s][1], stream=stream)
            batch.step(dt, stream=stream)
        stream.synchronize()
        for s in range(len(seqs)):
            assert np.array_equal(batch.slots[s][2].cpu().numpy(), outs[s][0].cpu().numpy()), (k, s)
            assert np.array_equal(batch.slots[s][3].cpu().numpy(), outs[s][1].cpu().numpy()), (k, s)
        rf, _ = ref.step(seqs[0].image[k], seqs[0].range[k], dt)
        e = np.abs(outs[0][0].cpu().numpy().astype(np.float64) - rf) * dt / dmu_ref[None]
        assert e.max() <= gu.FLOW_TOL_PX, (k, e.max())
    assert batch.launches_per_step() == 8 + 1 + 3          # eight one-wave propagation launches
    assert singles[0].kernels_per_step() == 7 + 1 + 3
    assert singles[1].kernels_per_step() == 1 + 1 + 2
    assert batch.status() in (sf.OK, sf.WARN_CFL)
