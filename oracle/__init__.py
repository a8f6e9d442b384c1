"""FP64 CPU oracle of the structure-flow predictor-update loop (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package.  The product library never loads it.  The arithmetic
lives in ``sf_oracle.c`` (plain C, double precision, compiled with
``-O2 -ffp-contract=off``); this module only builds it, loads it with ctypes and
marshals numpy arrays.  Every function cites the paper's section and equations
in the C source.

Parity pins: every function here is pinned by the ``-m "not gpu"`` tests
(closed forms, invariants, exact PDE solutions, brute force with exact
rational arithmetic).  The accuracy of the whole filter against real
ground-truth data (the paper's Urban Canyon numbers) is parity unpinned: the
dataset is not available, so the filter's error against analytic ground truth
is reported, not pinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "sf_oracle.c"
_LIB = _HERE / "libsf_oracle.so"

DOMINANT_LITERAL = 1
SOURCE_SPLIT = 2
IMU = 32

_lib = None


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (OpenMP over rows; no FMA contraction)."""
    if force or not _LIB.exists() or _LIB.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _LIB.with_suffix(f".so.tmp{os.getpid()}")
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               "-std=c11", "-Wall", "-o", str(tmp), str(_SRC), "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


_D = ctypes.POINTER(ctypes.c_double)
_U8 = ctypes.POINTER(ctypes.c_uint8)
_I = ctypes.POINTER(ctypes.c_int)


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(str(_LIB))
        i, d, vp = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
        L.sfo_set_threads.argtypes = [i]; L.sfo_set_threads.restype = i
        L.sfo_geometry.argtypes = [i, i, d, d, d, d, _D, _D, _D]
        L.sfo_image_model.argtypes = [i, i, _D, _D, _D, _D, _D, _D]
        L.sfo_invdepth_model.argtypes = [i, i, _D, _U8, _D, _D, _D, _D]
        L.sfo_propagate.argtypes = [i, i, i, i, _D, _D, _D, _D, _D, _D, _D, _D, _D]
        L.sfo_imu_step.argtypes = [i, i, d, _D, _D, _D, _D, _D]
        L.sfo_set_motion.argtypes = [vp, _D, _D]
        L.sfo_remap_pinhole.argtypes = [i, i, d, d, d, d, _D, i, i, _D, _D, _D, _D, _D]
        L.sfo_remap_equirect.argtypes = [i, i, d, d, d, d, _D, i, i, _D, _D, _D, _D]
        L.sfo_propagate.restype = d
        L.sfo_update.argtypes = [i, i, d, d, d, _D, _D, _D, _D, _D, _D, _U8, _D, _D, _D, _D]
        L.sfo_blend.argtypes = [i, d, d, _D, _U8, _D, _D]
        L.sfo_smooth.argtypes = [i, i, i, _D]
        L.sfo_downsample.argtypes = [i, i, _D, _D, _U8, _D, _D, _U8]
        L.sfo_upsample_add.argtypes = [i, i, _D, i, i, _D, _D]
        L.sfo_create.argtypes = [i, i, i, d, d, d, d, _I, _I, _D, d, i]
        L.sfo_create.restype = vp
        L.sfo_destroy.argtypes = [vp]
        L.sfo_reset.argtypes = [vp]
        L.sfo_step.argtypes = [vp, _D, _D, d, _D, _D]
        L.sfo_step.restype = d
        L.sfo_get_state.argtypes = [vp, i, _D, _D, _D, _D]
        L.sfo_set_state.argtypes = [vp, i, _D, _D, _D, _D, d]
        L.sfo_get_geometry.argtypes = [vp, i, _D, _D, _D]
        _lib = L
    return _lib


def set_threads(n: int) -> int:
    """Set the OpenMP thread count (n <= 0 keeps it); returns the count in use."""
    return lib().sfo_set_threads(int(n))


def _d(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _u8(a):
    assert a.dtype == np.uint8 and a.flags.c_contiguous
    return a.ctypes.data_as(_U8)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# stage functions (numpy in, numpy out; H x W scalar fields, H x W x 3 vectors)
# --------------------------------------------------------------------------

def geometry(H, W, fx, fy, cx, cy):
    """Pinhole-grid rays, tangent bases and spacing (Sec. 4.1, Eqs. 27-29)."""
    eta = np.empty((H, W, 3)); B = np.empty((H, W, 2, 3)); dmu = np.empty((H, W))
    lib().sfo_geometry(H, W, fx, fy, cx, cy, _d(eta), _d(B), _d(dmu))
    return eta, B, dmu


def level_intrinsics(fx, fy, cx, cy, level):
    """Intrinsics of pyramid level ``level`` (1-based): scaled by 2^(1-level)."""
    s = float(2 ** (level - 1))
    return fx / s, fy / s, cx / s, cy / s


def image_model(Y, B, dmu):
    """Weighted LS brightness model (Sec. 4.2, Eqs. 30-31): Yhat, d_beta, grad_eta."""
    Y = _f64(Y); H, W = Y.shape
    Yhat = np.empty((H, W)); db = np.empty((H, W, 2)); g = np.empty((H, W, 3))
    lib().sfo_image_model(H, W, _d(Y), _d(_f64(B)), _d(_f64(dmu)), _d(Yhat), _d(db), _d(g))
    return Yhat, db, g


def invdepth_model(rho, valid, B, dmu):
    """Occlusion-robust inverse-depth gradient (Sec. 4.3, Eqs. 32-34)."""
    rho = _f64(rho); H, W = rho.shape
    v = np.ascontiguousarray(valid, dtype=np.uint8)
    db = np.empty((H, W, 2)); g = np.empty((H, W, 3))
    lib().sfo_invdepth_model(H, W, _d(rho), _u8(v), _d(_f64(B)), _d(_f64(dmu)), _d(db), _d(g))
    return db, g


def propagate(w, rho, eta, B, dmu, N, dw=None, Y=None, flags=0, want_margin=False, imu=None):
    """N sub-iterations of the upwind scheme (Sec. 4.6, Eqs. 53-67).

    ``imu`` = (Omega, a) in frame units (rad/frame, m/frame^2), six numbers:
    with IMU in ``flags`` each sub-iteration ends with the inertial source step.
    Returns (w, dw, rho, Y, cfl[, margin]) -- copies; inputs are not modified.
    """
    w = _f64(w).copy(); rho = _f64(rho).copy()
    dw = None if dw is None else _f64(dw).copy()
    Y = None if Y is None else _f64(Y).copy()
    H, W = rho.shape
    margin = np.empty((H, W)) if want_margin else None
    m = None if imu is None else np.ascontiguousarray(np.asarray(imu, dtype=np.float64).reshape(6))
    cfl = lib().sfo_propagate(H, W, int(N), int(flags), _d(_f64(eta)), _d(_f64(B)), _d(_f64(dmu)),
                              _d(w), _d(dw), _d(rho), _d(Y), _d(margin), _d(m))
    out = (w, dw, rho, Y, cfl)
    return out + (margin,) if want_margin else out


def update(gamma123, eta, dmu, Yhat, gradY, rhohat, gradR, valid, Yref, rhoref, prior):
    """Per-pixel 3x3 least-squares update (Sec. 4.5, Eqs. 42-50)."""
    g1, g2, g3 = gamma123
    Yhat = _f64(Yhat); H, W = Yhat.shape
    x = np.empty((H, W, 3))
    lib().sfo_update(H, W, g1, g2, g3, _d(_f64(eta)), _d(_f64(dmu)), _d(Yhat), _d(_f64(gradY)),
                     _d(_f64(rhohat)), _d(_f64(gradR)), _u8(np.ascontiguousarray(valid, dtype=np.uint8)),
                     _d(_f64(Yref)), _d(_f64(rhoref)), _d(_f64(prior)), _d(x))
    return x


def blend(g4, g5, rhohat, valid, rho_pred):
    """Inverse-depth blend (Eqs. 51-52)."""
    rhohat = _f64(rhohat)
    out = np.empty_like(rhohat)
    lib().sfo_blend(rhohat.size, g4, g5, _d(rhohat), _u8(np.ascontiguousarray(valid, dtype=np.uint8)),
                    _d(_f64(rho_pred)), _d(out))
    return out


def smooth(f, S):
    """S passes of the 5x5 average filter (Sec. 4.5)."""
    f = _f64(f).copy(); H, W = f.shape[:2]
    lib().sfo_smooth(H, W, int(S), _d(f))
    return f


def downsample(Y, rho, valid):
    """One pyramid level down (2x2 mean; valid-mean of inverse depth)."""
    Y = _f64(Y); H, W = Y.shape
    Y2 = np.empty((H // 2, W // 2)); r2 = np.empty((H // 2, W // 2)); v2 = np.empty((H // 2, W // 2), np.uint8)
    lib().sfo_downsample(H, W, _d(Y), _d(_f64(rho)), _u8(np.ascontiguousarray(valid, dtype=np.uint8)),
                         _d(Y2), _d(r2), _u8(v2))
    return Y2, r2, v2


def upsample_add(wc, dw=None):
    """Eq. 26: bilinear x2 up-sampling of a coarse 3-vector field plus dw."""
    wc = _f64(wc); Hc, Wc = wc.shape[:2]
    H, W = 2 * Hc, 2 * Wc
    out = np.empty((H, W, 3))
    lib().sfo_upsample_add(Hc, Wc, _d(wc), H, W, _d(None if dw is None else _f64(dw)), _d(out))
    return out


# --------------------------------------------------------------------------
# remapping camera data onto the grid (readings R26, R27)
# --------------------------------------------------------------------------

def remap_pinhole(H, W, grid_K, R, cam_K, image, rng=None):
    """Grid (H x W, intrinsics grid_K = fx, fy, cx, cy) <- pinhole camera frame
    (cam_K, image/rng of any size); R = camera <- grid rotation.  Returns
    (image, range) on the grid (range None when rng is None)."""
    image = _f64(image); Hs, Ws = image.shape
    Rm = np.ascontiguousarray(np.asarray(R, dtype=np.float64).reshape(9))
    K = np.ascontiguousarray(np.asarray(cam_K, dtype=np.float64).reshape(4))
    oi = np.empty((H, W)); orng = np.empty((H, W)) if rng is not None else None
    lib().sfo_remap_pinhole(H, W, *[float(x) for x in grid_K], _d(Rm), Hs, Ws, _d(K), _d(image),
                            _d(None if rng is None else _f64(rng)), _d(oi), _d(orng))
    return oi, orng


def remap_equirect(H, W, grid_K, R, image, rng=None):
    """Grid <- equirectangular panorama (longitude across columns)."""
    image = _f64(image); Hs, Ws = image.shape
    Rm = np.ascontiguousarray(np.asarray(R, dtype=np.float64).reshape(9))
    oi = np.empty((H, W)); orng = np.empty((H, W)) if rng is not None else None
    lib().sfo_remap_equirect(H, W, *[float(x) for x in grid_K], _d(Rm), Hs, Ws, _d(image),
                             _d(None if rng is None else _f64(rng)), _d(oi), _d(orng))
    return oi, orng


# --------------------------------------------------------------------------
# propagation surrogate: one 3x3 convolution layer (plain definition)
# --------------------------------------------------------------------------

def conv3x3(x, w, b=None, relu=False):
    """y[n, i, j, co] = act(b[co] + sum_{dy, dx, ci} w[3 dy + dx, co, ci] x[n, i + dy - 1, j + dx - 1, ci])
    with zero padding, in float64.  x: [N, H, W, Cin]; w: [9, Cout, Cin]."""
    x = np.asarray(x, dtype=np.float64); w = np.asarray(w, dtype=np.float64)
    N, H, W, Cin = x.shape
    Cout = w.shape[1]
    xp = np.zeros((N, H + 2, W + 2, Cin))
    xp[:, 1:H + 1, 1:W + 1] = x
    y = np.zeros((N, H, W, Cout))
    for dy in range(3):
        for dx in range(3):
            y += xp[:, dy:dy + H, dx:dx + W, :] @ w[3 * dy + dx].T
    if b is not None:
        y += np.asarray(b, dtype=np.float64)
    return np.maximum(y, 0.0) if relu else y


# --------------------------------------------------------------------------
# whole filter
# --------------------------------------------------------------------------

@dataclass
class Params:
    """Filter parameters (same meaning as the C-ABI's ``sf_params``)."""
    fx: float
    fy: float
    cx: float
    cy: float
    iters: list = field(default_factory=lambda: [1])
    smooth: list = field(default_factory=lambda: [2])
    gamma: tuple = (1.0, 1.0, 1e-2, 1.0, 1.0)
    lambda_ref: float = 1.0
    flags: int = 0


class Filter:
    """The FP64 filter of Fig. 3 over an H x W image with L pyramid levels."""

    def __init__(self, H, W, L, params: Params):
        self.H, self.W, self.L, self.p = H, W, L, params
        it = (ctypes.c_int * 8)(*(list(params.iters) + [0] * 8)[:8])
        sm = (ctypes.c_int * 8)(*(list(params.smooth) + [0] * 8)[:8])
        g = (ctypes.c_double * 5)(*params.gamma)
        self._c = lib().sfo_create(H, W, L, params.fx, params.fy, params.cx, params.cy,
                                   it, sm, g, params.lambda_ref, params.flags)
        if not self._c:
            raise ValueError("invalid oracle filter configuration")
        self.last_cfl = 0.0

    def __del__(self):
        c = getattr(self, "_c", None)
        if c:
            lib().sfo_destroy(c)
            self._c = None

    def reset(self):
        lib().sfo_reset(self._c)

    def set_motion(self, omega=None, accel=None):
        """Camera angular velocity (rad/s) and linear acceleration (m/s^2), camera
        frame, for the next frames' predictions (used with IMU in the flags)."""
        om = None if omega is None else np.ascontiguousarray(np.asarray(omega, dtype=np.float64).reshape(3))
        ac = None if accel is None else np.ascontiguousarray(np.asarray(accel, dtype=np.float64).reshape(3))
        lib().sfo_set_motion(self._c, _d(om), _d(ac))

    def step(self, image, rng, dt):
        """One frame; returns (flow [3,H,W] rad/s, invdepth [H,W])."""
        flow = np.empty((3, self.H, self.W)); inv = np.empty((self.H, self.W))
        self.last_cfl = lib().sfo_step(self._c, _d(_f64(image)), _d(_f64(rng)), float(dt), _d(flow), _d(inv))
        return flow, inv

    def level_shape(self, h):
        return self.H >> h, self.W >> h

    def get_state(self, h):
        """Level h (0-based) state: dict of w, dw [H,W,3], rho, Yhat [H,W]."""
        Hh, Wh = self.level_shape(h)
        w = np.empty((Hh, Wh, 3)); dw = np.empty((Hh, Wh, 3)); r = np.empty((Hh, Wh)); y = np.empty((Hh, Wh))
        lib().sfo_get_state(self._c, h, _d(w), _d(dw), _d(r), _d(y))
        return dict(w=w, dw=dw, rho=r, Yhat=y)

    def set_state(self, h, w=None, dw=None, rho=None, Yhat=None, dt_prev=1.0):
        lib().sfo_set_state(self._c, h, _d(None if w is None else _f64(w)), _d(None if dw is None else _f64(dw)),
                            _d(None if rho is None else _f64(rho)), _d(None if Yhat is None else _f64(Yhat)),
                            float(dt_prev))

    def geometry(self, h):
        Hh, Wh = self.level_shape(h)
        eta = np.empty((Hh, Wh, 3)); B = np.empty((Hh, Wh, 2, 3)); dmu = np.empty((Hh, Wh))
        lib().sfo_get_geometry(self._c, h, _d(eta), _d(B), _d(dmu))
        return eta, B, dmu
