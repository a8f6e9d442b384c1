"""Helpers shared by the GPU parity tests: seeded inputs and error measures.

Every input is made float32 first; the oracle receives those exact values in
float64, so both sides compute from identical data.
"""
import numpy as np

import oracle
from paper_2406_18031_b300 import sf

FLOW_TOL_PX = 1e-4        # px/frame, max-abs per stage
RHO_TOL = 1e-5            # inverse depth, absolute (values 0.02 .. 1)
Y_TOL = 1e-5              # brightness, absolute (values in [0, 1])
DRIFT_TOL = 1e-3          # relative L2 after 100 frames


def level_grid(H1, W1, fx, fy, cx, cy, level):
    """(sf.CGrid, oracle geometry) of pyramid level ``level`` (1-based)."""
    s = 2 ** (level - 1)
    H, W = H1 // s, W1 // s
    ifx, ify, icx, icy = oracle.level_intrinsics(fx, fy, cx, cy, level)
    g = sf.grid(H, W, ifx, ify, icx, icy)
    eta, B, dmu = oracle.geometry(H, W, ifx, ify, icx, icy)
    return g, eta, B, dmu


def smooth_field(rng, H, W, n_waves=4, scale=1.0):
    """Smooth random scalar field in [-scale, scale]-ish."""
    i, j = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    out = np.zeros((H, W))
    for _ in range(n_waves):
        k = rng.uniform(0.02, 0.25, size=2) * rng.choice([-1, 1], size=2)
        out += rng.uniform(0.3, 1.0) * np.sin(k[0] * i + k[1] * j + rng.uniform(0, 6.3))
    return scale * out / n_waves


def flow_field(rng, H, W, dmu, max_px, with_step=True):
    """Structure flow in rad/frame whose tangential part reaches ~max_px px/frame,
    with an occlusion-like step discontinuity across a random line."""
    w = np.stack([smooth_field(rng, H, W), smooth_field(rng, H, W), 0.3 * smooth_field(rng, H, W)], -1)
    if with_step:
        i, j = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
        a, b = rng.normal(size=2)
        side = (a * (i - H / 2) + b * (j - W / 2)) > 0
        w[side] = w[side] * -0.6 + 0.2
    w *= max_px / max(np.abs(w[..., :2]).max(), 1e-12)
    return (w * dmu[..., None]).astype(np.float32)


def cfl_scaled(w, eta, B, dmu, max_px):
    """Scale a flow field (rad/frame) so its largest pixel speed (Eq. 54:
    B^T P w / dmu) is max_px."""
    Pw = w - eta * np.einsum("hwc,hwc->hw", eta, w)[..., None]
    sp = np.abs(np.einsum("hwkc,hwc->hwk", B, Pw)) / dmu[..., None]
    return (w * (max_px / max(sp.max(), 1e-30))).astype(np.float32)


def f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def px_err(w_gpu, w_ref, dmu):
    """max over pixels and components of |w_gpu - w_ref| / dmu (px/frame)."""
    return float((np.abs(np.asarray(w_gpu, np.float64) - w_ref) / dmu[..., None]).max())


def rel_l2(a, b):
    a = np.asarray(a, np.float64); b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def oracle_level_data(image, rng_, levels, lambda_ref=1.0):
    """Level data (Y, rho-hat, valid) for levels 1..levels from float32 inputs."""
    Y = image.astype(np.float64)
    lam = rng_.astype(np.float64)
    valid = (np.isfinite(lam) & (lam > 0)).astype(np.uint8)
    with np.errstate(divide="ignore", invalid="ignore"):
        rho = np.where(valid > 0, lambda_ref / lam, 0.0)
    out = [(Y, rho, valid)]
    for _ in range(1, levels):
        Y, rho, valid = oracle.downsample(Y, rho, valid)
        out.append((Y, rho, valid))
    return out


def bf16_round(a):
    """float32 -> the nearest bfloat16 (ties to even), returned as float32."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def bf16_bits(a):
    """float32 values exactly representable in bfloat16 -> their uint16 bit patterns."""
    return (np.ascontiguousarray(a, dtype=np.float32).view(np.uint32) >> 16).astype(np.uint16)
