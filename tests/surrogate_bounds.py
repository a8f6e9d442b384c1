"""Element-wise tolerance for the surrogate's training gradients (float32
CUDA path against the float64 oracle).

Both sides store bfloat16 at the same points (features, weights, hidden
activations, output gradient, input gradients) and accumulate every sum of
products; they differ by float32 rounding and by the few bfloat16 stores (and
ReLU decisions) that land on different sides of a rounding boundary (of zero)
because the two sums feeding them differ in their last float32 bits.  Each
such isolated difference moves a weight gradient dW[tap, co, ci] = sum over
pixels of dy[p, co] x[p + tap, ci] by at most 2^-7 (one bfloat16 ulp,
relative) of the |.|-weighted sum of the same products, and float32
accumulation over n pixels by at most n 2^-23 of it.  The tolerance is the
sum of the two, per parameter; tests/test_oracle_surrogate.py checks that it
holds for a float32 restatement of the network and that a transposed channel
block or a shifted tap exceeds it in most elements."""
import numpy as np

from oracle import surrogate as S

BF = 2.0 ** -7          # one bfloat16 ulp, relative to the value, at most


def oracle_gradients_and_tolerance(x0, params, t):
    """x0: features [n, H, W, 16] (float64, not yet rounded); params: flat
    float32 parameters; t: target in the network's units.  Returns (loss,
    gradient, tolerance): the oracle's surrogate.loss_and_grads(..., q=bf16)
    and, per parameter, (2^-7 + n_px 2^-23) x sum of |dy| |x| over the
    products of that parameter's gradient (the bias: sum of |dy|)."""
    q = S.bf16
    loss, grads = S.loss_and_grads(x0, params, t, q=q)
    acts, out = S.forward(x0, params, q=q)
    layers = S.split_params(params)
    n_px = out.shape[0] * out.shape[1] * out.shape[2]
    dy = np.zeros_like(out)
    dy[..., :4] = 2.0 * (out - t)[..., :4] / (4 * n_px)
    dy = q(dy)
    mags = [None] * 4
    for l in range(3, -1, -1):
        mags[l] = S.conv3x3_wgrad(np.abs(acts[l]), np.abs(dy))
        if l == 0:
            break
        dx = q(S.conv3x3_dgrad(dy, q(layers[l][0])))
        dy = np.where(acts[l] > 0, dx, 0.0)
    mag = np.concatenate([np.concatenate([m[0].ravel(), m[1]]) for m in mags])
    return loss, grads, (BF + n_px * 2.0 ** -23) * mag
