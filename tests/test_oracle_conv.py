"""Pins of the oracle's 3x3 convolution layer (the surrogate's building block):
per-channel cross-correlation from scipy, the identity kernel, zero padding."""
import numpy as np
from scipy.signal import correlate2d


def test_conv_matches_scipy_cross_correlation(oracle):
    rng = np.random.default_rng(1)
    N, H, W, Cin, Cout = 2, 7, 9, 3, 4
    x = rng.normal(size=(N, H, W, Cin))
    w = rng.normal(size=(9, Cout, Cin))
    b = rng.normal(size=Cout)
    y = oracle.conv3x3(x, w, b)
    for n in range(N):
        for co in range(Cout):
            ref = np.full((H, W), b[co])
            for ci in range(Cin):
                k = w[:, co, ci].reshape(3, 3)
                ref += correlate2d(x[n, :, :, ci], k, mode="same", boundary="fill", fillvalue=0.0)
            np.testing.assert_allclose(y[n, :, :, co], ref, rtol=1e-12, atol=1e-12)


def test_identity_kernel_and_relu(oracle):
    rng = np.random.default_rng(2)
    x = rng.normal(size=(1, 5, 6, 8))
    w = np.zeros((9, 8, 8)); w[4] = np.eye(8)
    np.testing.assert_array_equal(oracle.conv3x3(x, w), x)
    np.testing.assert_array_equal(oracle.conv3x3(x, w, relu=True), np.maximum(x, 0))


def test_zero_padding_counts_the_taps_inside(oracle):
    x = np.ones((1, 4, 5, 1)); w = np.ones((9, 1, 1))
    y = oracle.conv3x3(x, w)[0, :, :, 0]
    assert y[0, 0] == 4 and y[0, 2] == 6 and y[1, 1] == 9 and y[3, 4] == 4
