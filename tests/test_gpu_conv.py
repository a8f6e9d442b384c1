"""Parity of the tensor-core 3x3 convolution (sf_conv3x3) with the oracle.

Inputs and weights are bfloat16 values; the oracle convolves exactly those
values in float64.  FP32 accumulation of 9 Cin bf16 products: the float32
output is within 1e-5 of the sum of |x w| per output (about 200 float32
roundings of a partial sum); the bfloat16 output within one bf16 ulp of the
oracle's value rounded to bfloat16, plus that float32 error (the float32 sum
may sit on the other side of a rounding boundary, or of zero under ReLU)."""
import numpy as np
import pytest

import oracle
from oracle import surrogate as oracle_surrogate
from paper_2406_18031_b300 import sf
from tests import gpu_util as gu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _bf16_tensor(a):
    bits = gu.bf16_bits(a).astype(np.int16)
    return torch.from_numpy(bits).cuda().view(torch.bfloat16)


def _case(N, H, W, Cin, Cout, relu, seed):
    rng = np.random.default_rng(seed)
    x = gu.bf16_round(rng.normal(size=(N, H, W, Cin)).astype(np.float32))
    w = gu.bf16_round((rng.normal(size=(9, Cout, Cin)) / np.sqrt(9 * Cin)).astype(np.float32))
    b = rng.normal(size=Cout).astype(np.float32) * 0.1
    y = torch.empty((N, H, W, Cout), dtype=torch.bfloat16, device="cuda")
    y32 = torch.empty((N, H, W, Cout), dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    sf.conv3x3(_bf16_tensor(x), _bf16_tensor(w), torch.from_numpy(b).cuda(), relu, y, y32, st)
    torch.cuda.synchronize()
    ref = oracle.conv3x3(x, w, b, relu)
    mag = oracle.conv3x3(np.abs(x), np.abs(w), np.abs(b))
    got32 = y32.cpu().numpy()
    assert np.all(np.abs(got32 - ref) <= 1e-5 * mag + 1e-7), np.abs(got32 - ref).max()
    got = y.float().cpu().numpy()
    # one bf16 ulp of the value plus the float32 accumulation error (which can
    # also move a value across zero under ReLU)
    tol = np.abs(gu.bf16_round(ref.astype(np.float32))) * 2.0 ** -7 + 1e-5 * mag + 1e-7
    assert np.all(np.abs(got - gu.bf16_round(ref.astype(np.float32))) <= tol)
    assert int(st.item()) == 0


@pytest.mark.parametrize("Cin,Cout", [(16, 16), (16, 32), (32, 16), (32, 32)])
@pytest.mark.parametrize("relu", [False, True])
def test_conv_small_ragged(Cin, Cout, relu):
    # two tiles per row, the second 72 pixels wide
    _case(2, 5, 200, Cin, Cout, relu, seed=Cin + Cout + relu)


def test_conv_larger_frame():
    _case(1, 64, 512, 32, 32, True, seed=3)


def test_conv_narrow_image():
    _case(3, 9, 37, 16, 32, False, seed=4)


def test_bounded_wait_gives_up_and_leaves_the_device_usable():
    # a tile whose MMAs are never issued: its completion wait cannot succeed;
    # the kernel must report the timeout, free its tensor memory and return
    assert sf.lib().sf_selftest_conv_timeout(None) == sf.ETIMEOUT
    _case(1, 3, 130, 16, 16, True, seed=5)       # and the next convolution still works


def test_binding_rejects_wrong_buffers_before_the_call():
    x = torch.zeros((1, 8, 8, 16), dtype=torch.bfloat16, device="cuda")
    w = torch.zeros((9, 32, 16), dtype=torch.bfloat16, device="cuda")
    y = torch.empty((1, 8, 8, 32), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(ValueError, match="w: expected"):
        sf.conv3x3(x, w[:, :, :8].contiguous(), y=y)                   # Cin of w differs from x's
    with pytest.raises(ValueError, match="y: expected"):
        sf.conv3x3(x, w, y=y.float())                                  # float32 tensor as the bf16 output
    with pytest.raises(ValueError, match="y32: expected 2048"):
        sf.conv3x3(x, w, y32=torch.empty((1, 8, 7, 32), device="cuda"))
    with pytest.raises(ValueError, match="bias: expected"):
        sf.conv3x3(x, w, torch.zeros(16, device="cuda"), y=y)
    with pytest.raises(ValueError, match="status: expected"):
        sf.conv3x3(x, w, y=y, status=torch.zeros(1, dtype=torch.int64, device="cuda"))
    sf.conv3x3(x, w, y=y)                                              # the right ones still work
    torch.cuda.synchronize()
    assert float(y.float().abs().max()) == 0.0


@pytest.mark.parametrize("Cin,Cout", [(16, 32), (32, 32), (32, 16)])
def test_weight_gradient_element_by_element(Cin, Cout):
    # sf_conv3x3_wgrad: dW[tap, co, ci] = sum_p dy[p, co] x[p + tap, ci] over
    # N x H x W pixels (two frames, rows of two tiles, the second ragged).
    # The bf16 x bf16 products are exact in float32; float32 accumulation
    # over n pixels is within n 2^-23 of the sum of |products|.  Channel
    # means that differ per channel make every (co, ci) entry distinct, so
    # a transposed block or a shifted tap cannot hide under the tolerance.
    N, H, W = 2, 7, 200
    rng = np.random.default_rng(Cin * 3 + Cout)
    x = gu.bf16_round((rng.normal(size=(N, H, W, Cin)) + 0.2 * np.arange(Cin) - 1.0).astype(np.float32))
    dy = gu.bf16_round((rng.normal(size=(N, H, W, Cout)) * 0.5 + 0.1 * (np.arange(Cout) - 8)).astype(np.float32))
    dw = torch.full((9, Cout, Cin), float("nan"), device="cuda")
    db = torch.full((Cout,), float("nan"), device="cuda")
    sf.conv3x3_wgrad(_bf16_tensor(x), _bf16_tensor(dy), dw, db)
    torch.cuda.synchronize()
    ref_w, ref_b = oracle_surrogate.conv3x3_wgrad(x, dy)
    mag_w, mag_b = oracle_surrogate.conv3x3_wgrad(np.abs(x), np.abs(dy))
    gam = N * H * W * 2.0 ** -23
    got_w, got_b = dw.cpu().numpy(), db.cpu().numpy()
    assert np.all(np.abs(got_w - ref_w) <= gam * mag_w)
    assert np.all(np.abs(got_b - ref_b) <= gam * mag_b)
    # the tolerance separates neighbouring taps and swapped channels
    assert (np.abs(np.roll(ref_w, 1, axis=0) - ref_w) > gam * mag_w).mean() > 0.9
    assert (np.abs(np.swapaxes(ref_w[:, :16, :16], 1, 2) - ref_w[:, :16, :16]) > gam * mag_w[:, :16, :16]).mean() > 0.8


def test_weight_gradient_called_twice_overwrites():
    # the entry point overwrites its outputs (the kernel adds into zeroed buffers)
    rng = np.random.default_rng(7)
    x = gu.bf16_round(rng.normal(size=(1, 3, 130, 16)).astype(np.float32))
    dy = gu.bf16_round(rng.normal(size=(1, 3, 130, 16)).astype(np.float32))
    dw = torch.empty((9, 16, 16), device="cuda")
    db = torch.empty((16,), device="cuda")
    sf.conv3x3_wgrad(_bf16_tensor(x), _bf16_tensor(dy), dw, db)
    first = dw.clone(), db.clone()
    sf.conv3x3_wgrad(_bf16_tensor(x), _bf16_tensor(dy), dw, db)
    torch.cuda.synchronize()
    assert torch.allclose(dw, first[0], rtol=1e-6, atol=1e-6) and torch.allclose(db, first[1], rtol=1e-6, atol=1e-6)
