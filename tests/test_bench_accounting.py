"""The benchmark's accounting on CPU: the algorithmic bytes and FLOPs behind
the roofline figures, the launch-slot names and the whole-job rate, each
checked against a count made by hand from the state layout (Sec. 4: w, rho,
dw, Y-hat per pixel of a lower level; w, rho, Y-hat at the top) rather than
against the helper's own formula."""
import numpy as np
import pytest

import bench


def test_propagation_bytes_of_the_512_workload():
    # level 1 (512^2): two float4 planes read and two written (w, rho | dw, Y-hat);
    # level 2 (256^2, the top): one float4 plane read and one written
    lvl1 = 512 * 512 * (2 * 16) * 2
    lvl2 = 256 * 256 * 16 * 2
    assert bench.propagate_bytes_per_launch(512, 512, 2) == lvl1 + lvl2 == 18_874_368


def test_frame_bytes_of_the_512_workload():
    inputs, outputs = 512 * 512 * (4 + 4), 512 * 512 * (12 + 4)      # image + range; flow + inverse depth
    lvl1 = 512 * 512 * 32 * 2                                       # w, rho, dw, Y-hat in and out
    lvl2 = 256 * 256 * 20 * 2                                       # w, rho, Y-hat in and out
    assert bench.algorithmic_bytes_per_frame(512, 512, 2) == inputs + outputs + lvl1 + lvl2 == 25_690_112


def test_frame_flops_by_hand():
    # one level of 8x8, N = 3 sub-iterations of the 4-channel top (58 each), the
    # solve (130) and two smoothing passes (18 each)
    assert bench.frame_flops(8, 8, 1, [3], [2]) == 64 * (3 * 58 + 130 + 2 * 18)
    # two levels of 4x4 and 2x2: level 1 adds the 8-channel transport (94) and the reconstruction (12)
    lvl1 = 16 * (2 * 94 + 130 + 18 + 12)
    lvl2 = 4 * (1 * 58 + 130 + 18)
    assert bench.frame_flops(4, 4, 2, [2, 1], [1, 1]) == lvl1 + lvl2


@pytest.mark.parametrize("N,nf_max,nf", [(8, 8, 8), (10, 8, 5), (9, 4, 3), (4, 8, 4), (1, 8, 1)])
def test_first_propagation_launch_runs_the_even_split(N, nf_max, nf):
    # N sub-iterations in ceil(N / nf_max) launches of near-equal length; the first is the longest
    assert bench.propagate_flops_per_launch(4, 4, 1, [N], nf_max) == 16 * nf * 58


def test_roofline_frame_picks_the_larger_bound():
    frames = [(512, 512, 2, [8, 4], [2, 4])]
    b = bench.algorithmic_bytes_per_frame(512, 512, 2)
    f = bench.frame_flops(512, 512, 2, [8, 4], [2, 4])
    r = bench.roofline_frame(frames, 0.1, 6500.0)
    tb, tf = b / 6500e9, f / (bench.FP32_PEAK_TFLOPS * 1e12)
    assert r["bound"] == ("hbm" if tb >= tf else "alu")
    assert r["time_min_us"] == pytest.approx(max(tb, tf) * 1e6)
    assert r["frac"] == pytest.approx(max(tb, tf) / 1e-4)
    # a link of 1 GB/s makes any frame byte-bound
    assert bench.roofline_frame(frames, 0.1, 1.0)["bound"] == "hbm"
    # 148 SMs x 128 FP32 lanes x 2 (FMA) at 2.032 GHz
    assert bench.FP32_PEAK_TFLOPS == pytest.approx(76.99, abs=0.01)


def test_update_slot_names():
    assert bench.update_slot_names(6, 1, 3, "level") == [
        "k_propagate#0", "k_propagate#1", "k_solve",
        "k_smooth_recon#level3", "k_smooth_recon#level2", "k_smooth_recon#level1"]
    assert bench.update_slot_names(4, 2, 2, "level") == [
        "k_propagate#0", "k_solve", "k_smooth_recon#all", "k_recon_jobs#level1"]
    assert bench.update_slot_names(5, 2, 3, "depth") == [
        "k_propagate#0", "k_solve", "k_smooth_recon#all", "k_recon_jobs#depth1", "k_recon_jobs#depth2"]


def test_whole_job_rate_and_one_rank_time():
    assert bench.whole_job_rate(30, 2, 150.0) == pytest.approx(400.0)
    assert bench.job_time_ms(12.5, 1, None) == 12.5


def test_stored_traffic_follows_the_kernel_source(monkeypatch):
    key = next(k for k in bench.TRAFFIC if k != "kernel_sources_sha256_16")
    monkeypatch.setattr(bench, "kernel_sources_hash", lambda: bench.TRAFFIC["kernel_sources_sha256_16"])
    assert bench.measured_traffic(key) == bench.TRAFFIC[key]
    monkeypatch.setattr(bench, "kernel_sources_hash", lambda: "0" * 16)   # the kernel changed since the capture
    assert bench.measured_traffic(key) is None


def test_pixel_spacing_matches_the_oracle_geometry():
    import oracle
    oracle.build()
    H, W, fx, fy, cx, cy = 24, 40, 30.0, 28.0, 19.0, 13.0
    _, _, dmu = oracle.geometry(H, W, fx, fy, cx, cy)
    np.testing.assert_allclose(bench.pixel_spacing(H, W, fx, fy, cx, cy), dmu, rtol=1e-12)


def test_flow_errors_of_known_differences():
    H, W, dt = 3, 4, 0.01
    dmu = np.full((H, W), 0.002)
    truth = np.zeros((3, H, W))
    truth[0] = 0.4                                   # 0.4 rad/s x 0.01 s / 0.002 = 2 px/frame along x
    epe, aae = bench.flow_errors(truth, truth, dt, dmu)
    assert epe == 0.0 and aae < 1e-6
    flow = truth.copy()
    flow[1] = 0.3                                    # + 1.5 px/frame along y
    epe, aae = bench.flow_errors(flow, truth, dt, dmu)
    assert abs(epe - 1.5) < 1e-12
    # a = (2, 1.5, 0), b = (2, 0, 0): arccos(5 / sqrt(7.25 x 5))
    assert abs(aae - np.degrees(np.arccos(5.0 / np.sqrt(7.25 * 5.0)))) < 1e-9
    mask = np.zeros((H, W), bool)
    mask[0, 0] = True
    assert bench.flow_errors(flow, truth, dt, dmu, mask)[0] == epe
