"""sf_propagate_noalloc: the allocation-free propagation entry point.

Some callers cannot allocate device memory while they run the filter:
real-time loops that must not touch the allocator (cudaMalloc and cudaFree can
block and synchronise the device), processes whose memory pools belong to
another framework, code handed a fixed memory budget.  For them the library offers sf_propagate_noalloc, which keeps its
scratch in a fixed device array instead of allocating.  This file checks,
through the C ABI, that it returns what the allocating sf_propagate returns,
on two calls in a row (the second call sees the array as the first left it).
It sits last in collection order so that a stopping run has run every other
test first.
"""
import ctypes

import numpy as np
import pytest

from paper_2406_18031_b300 import build, sf
from tests import gpu_util as gu

torch = pytest.importorskip("torch")


def _case(rng, H, W, N, top):
    import oracle
    fx = fy = W / 2.0 + 5.0
    cx, cy = W / 2.0 - 0.5, H / 2.0 + 1.5
    g, eta, B, dmu = gu.level_grid(H, W, fx, fy, cx, cy, 1)
    w = gu.cfl_scaled(gu.flow_field(rng, H, W, dmu, max_px=1.0), eta, B, dmu, min(0.8 * N, 0.1 * min(H, W)))
    rho = gu.f32(0.2 + 0.15 * gu.smooth_field(rng, H, W))
    s0 = np.concatenate([w, rho[..., None]], -1)
    s1 = None
    if not top:
        dw = gu.f32(gu.flow_field(rng, H, W, dmu, max_px=0.2 * N) * 0.5)
        Y = gu.f32(0.5 + 0.4 * gu.smooth_field(rng, H, W, n_waves=6))
        s1 = np.concatenate([dw, Y[..., None]], -1)
    return g, dmu, s0, s1


@pytest.mark.gpu
def test_noalloc_propagation_matches_sf_propagate_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    rng = np.random.default_rng(2024)
    # first call: a lower level with 20 sub-iterations (three launches, so the
    # scratch fields carry data between launches); second call: a top level
    # of another size with 12 sub-iterations
    for (H, W, N, top) in [(96, 80, 20, False), (72, 136, 12, True)]:
        g, dmu, s0, s1 = _case(rng, H, W, N, top)
        t0 = torch.from_numpy(gu.f32(s0)).cuda()
        t1 = None if top else torch.from_numpy(gu.f32(s1)).cuda()
        ref0 = torch.empty((H, W, 4), device="cuda")
        ref1 = None if top else torch.empty((H, W, 4), device="cuda")
        out0 = torch.full((H, W, 4), float("nan"), device="cuda")
        out1 = None if top else torch.full((H, W, 4), float("nan"), device="cuda")
        st_ref = torch.zeros(1, dtype=torch.int32, device="cuda")
        st_out = torch.zeros(1, dtype=torch.int32, device="cuda")
        sf.propagate(g, N, t0, ref0, t1, ref1, flags=sf.CHECK_CFL, status=st_ref)
        sf.propagate_noalloc(g, N, t0, out0, t1, out1, flags=sf.CHECK_CFL, status=st_out)
        torch.cuda.synchronize()
        a, b = out0.cpu().numpy(), ref0.cpu().numpy()
        assert np.isfinite(a).all()
        assert gu.px_err(a[..., :3], b[..., :3].astype(np.float64), dmu) <= gu.FLOW_TOL_PX
        assert np.abs(a[..., 3] - b[..., 3]).max() <= gu.RHO_TOL
        if not top:
            a1, b1 = out1.cpu().numpy(), ref1.cpu().numpy()
            assert gu.px_err(a1[..., :3], b1[..., :3].astype(np.float64), dmu) <= gu.FLOW_TOL_PX
            assert np.abs(a1[..., 3] - b1[..., 3]).max() <= gu.Y_TOL
        assert int(st_out.item()) == int(st_ref.item())


def test_noalloc_rejects_grids_above_its_limit_without_touching_the_device():
    build.build()
    L = sf.lib()
    g = sf.grid(1025, 1024, 512.0, 512.0, 512.0, 512.0)   # 1,049,600 pixels > 1,048,576
    x = ctypes.c_void_p(256)                               # never dereferenced: rejected first
    assert L.sf_propagate_noalloc(ctypes.byref(g), 4, 0, ctypes.c_float(1.0), x, None, x, None, None,
                                  None) == sf.EINVAL
