"""ctypes binding of libsf (include/sf.h): argument marshalling only.

Every step of the filter runs in the library's CUDA kernels; this module only
converts torch tensors and Python values into the C ABI's pointers and
structs.  There is no CPU path: if the library cannot be loaded, or a CUDA
device is missing, calls raise.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field
from pathlib import Path

import numpy as np

_PKG = Path(__file__).resolve().parent
LIB_PATH = _PKG / "libsf.so"

MAX_LEVELS = 4
OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENONFINITE, WARN_CFL = 0, -1, -2, -3, -4, -5, 1
DOMINANT_LITERAL, SOURCE_SPLIT, CHECK_CFL, CHECK_FINITE, AUTOTUNE, IMU = 1, 2, 4, 8, 16, 32


class SFError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {strerror(code)} ({code})")
        self.code = code


class CParams(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("iters", ctypes.c_int * MAX_LEVELS), ("max_flow", ctypes.c_float),
                ("smooth_iters", ctypes.c_int * MAX_LEVELS), ("gamma", ctypes.c_float * 5),
                ("lambda_ref", ctypes.c_float), ("flags", ctypes.c_int), ("nf_max", ctypes.c_int),
                ("update_mode", ctypes.c_int), ("solve_tile", ctypes.c_int)]


class CGrid(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int), ("W", ctypes.c_int), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float)]


_lib = None

EXPORTS = ["sf_params_default", "sf_create", "sf_reset", "sf_step", "sf_step_host", "sf_submit_host", "sf_wait_host", "sf_status", "sf_get_state",
           "sf_set_state", "sf_kernels_per_step", "sf_nf_max", "sf_update_mode", "sf_solve_tile", "sf_set_motion", "sf_propagate_imu", "sf_profile", "sf_profile_read", "sf_destroy", "sf_strerror", "sf_propagate", "sf_propagate_noalloc",
           "sf_update", "sf_reconstruct", "sf_batch_create", "sf_batch_buffers", "sf_batch_step",
           "sf_batch_status", "sf_batch_launches_per_step", "sf_batch_nf_max", "sf_batch_update_mode", "sf_batch_solve_tile", "sf_batch_motion", "sf_batch_profile",
           "sf_batch_profile_read",
           "sf_batch_destroy", "sf_remap_pinhole", "sf_remap_equirect", "sf_conv3x3", "sf_conv3x3_wgrad", "sf_selftest_conv_timeout", "sf_selftest_net_timeout", "sf_surrogate_create",
           "sf_surrogate_destroy", "sf_surrogate_num_params", "sf_surrogate_params", "sf_surrogate_grads",
           "sf_surrogate_forward", "sf_surrogate_forward_layered", "sf_surrogate_train_step", "sf_surrogate_propagate", "sf_set_surrogate",
           "sf_batch_set_surrogate", "sf_set_surrogate_threshold", "sf_batch_set_surrogate_threshold",
           "sf_surrogate_stats", "sf_batch_surrogate_stats", "sf_set_trace"]


def lib():
    """Load libsf.so (built by ``paper_2406_18031_b300.build``); raises if absent."""
    global _lib
    if _lib is None:
        if not LIB_PATH.exists():
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2406_18031_b300.build`")
        L = ctypes.CDLL(str(LIB_PATH))
        i, f, vp = ctypes.c_int, ctypes.c_float, ctypes.c_void_p
        P = ctypes.POINTER
        L.sf_params_default.argtypes = [P(CParams), i, i, i]
        L.sf_create.argtypes = [i, i, i, P(CParams), P(vp)]
        L.sf_reset.argtypes = [vp]
        L.sf_step.argtypes = [vp, vp, vp, f, vp, vp, vp]
        L.sf_step_host.argtypes = [vp, vp, vp, f, vp, vp, vp]
        L.sf_submit_host.argtypes = [vp, vp, vp, f, vp, vp, vp, P(ctypes.c_longlong)]
        L.sf_wait_host.argtypes = [vp, ctypes.c_longlong]
        L.sf_status.argtypes = [vp]
        L.sf_get_state.argtypes = [vp, i, vp, P(f), vp]
        L.sf_set_state.argtypes = [vp, i, vp, f, vp]
        L.sf_kernels_per_step.argtypes = [vp]
        L.sf_nf_max.argtypes = [vp]
        L.sf_update_mode.argtypes = [vp]
        L.sf_solve_tile.argtypes = [vp]
        L.sf_profile.argtypes = [vp, i]
        L.sf_profile_read.argtypes = [vp, P(f), P(i), i]
        L.sf_destroy.argtypes = [vp]
        L.sf_destroy.restype = None
        L.sf_strerror.argtypes = [i]
        L.sf_strerror.restype = ctypes.c_char_p
        L.sf_propagate.argtypes = [P(CGrid), i, i, f, vp, vp, vp, vp, vp, vp]
        L.sf_propagate_imu.argtypes = [P(CGrid), i, i, f, P(f), vp, vp, vp, vp, vp, vp]
        L.sf_set_motion.argtypes = [vp, P(f), P(f), vp]
        L.sf_remap_pinhole.argtypes = [P(CGrid), P(f), i, i, P(f), vp, vp, vp, vp, vp]
        L.sf_conv3x3.argtypes = [i, i, i, i, i, vp, vp, vp, i, vp, vp, vp, vp]
        L.sf_conv3x3_wgrad.argtypes = [i, i, i, i, i, vp, vp, vp, vp, vp]
        L.sf_selftest_conv_timeout.argtypes = [vp]
        L.sf_selftest_net_timeout.argtypes = [vp]
        L.sf_surrogate_create.argtypes = [ctypes.c_ulonglong, P(vp)]
        L.sf_surrogate_destroy.argtypes = [vp]
        L.sf_surrogate_destroy.restype = None
        L.sf_surrogate_num_params.argtypes = [vp]
        L.sf_surrogate_params.argtypes = [vp, P(f), i]
        L.sf_surrogate_grads.argtypes = [vp, P(f)]
        L.sf_surrogate_forward.argtypes = [vp, P(CGrid), i, vp, vp, vp]
        L.sf_surrogate_forward_layered.argtypes = [vp, P(CGrid), i, vp, vp, vp]
        L.sf_surrogate_train_step.argtypes = [vp, P(CGrid), i, vp, vp, f, P(f), vp]
        L.sf_surrogate_propagate.argtypes = [vp, P(CGrid), i, i, vp, vp, f, P(f), P(i), vp]
        L.sf_set_surrogate.argtypes = [vp, vp]
        L.sf_batch_set_surrogate.argtypes = [vp, vp]
        L.sf_set_trace.argtypes = [i]
        L.sf_set_surrogate_threshold.argtypes = [vp, f]
        L.sf_batch_set_surrogate_threshold.argtypes = [vp, i, f]
        L.sf_surrogate_stats.argtypes = [vp, P(f), P(i)]
        L.sf_batch_surrogate_stats.argtypes = [vp, P(f), P(i), i]
        L.sf_remap_equirect.argtypes = [P(CGrid), P(f), i, i, vp, vp, vp, vp, vp]
        L.sf_batch_motion.argtypes = [vp, i, P(vp)]
        L.sf_batch_create.argtypes = [i, P(i), P(i), P(i), P(CParams), P(vp)]
        L.sf_batch_buffers.argtypes = [vp, i, P(vp), P(vp), P(vp), P(vp)]
        L.sf_batch_step.argtypes = [vp, f, vp]
        L.sf_batch_status.argtypes = [vp]
        L.sf_batch_launches_per_step.argtypes = [vp]
        L.sf_batch_nf_max.argtypes = [vp]
        L.sf_batch_update_mode.argtypes = [vp]
        L.sf_batch_solve_tile.argtypes = [vp]
        L.sf_batch_profile.argtypes = [vp, i]
        L.sf_batch_profile_read.argtypes = [vp, P(f), P(i), i]
        L.sf_batch_destroy.argtypes = [vp]
        L.sf_batch_destroy.restype = None
        L.sf_propagate_noalloc.argtypes = [P(CGrid), i, i, f, vp, vp, vp, vp, vp, vp]
        L.sf_update.argtypes = [P(CGrid), i, i, i, i, P(f), f, vp, vp, i, i, vp, vp, vp, vp, vp, vp, vp, vp]
        L.sf_reconstruct.argtypes = [i, P(CGrid), P(vp), P(vp), f, vp, vp, i, vp, vp]
        _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().sf_strerror(int(code)).decode()


def _check(code, what):
    if code < 0:
        raise SFError(code, what)
    return code


def _ptr(t, itemsize=4):
    """Device pointer of a CUDA tensor (or None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous() or t.dtype.itemsize != itemsize:
        raise ValueError(f"expected a contiguous {8 * itemsize}-bit tensor")
    return ctypes.c_void_p(t.data_ptr())


def _tptr(t, dtype, n, what):
    """Device pointer of a contiguous CUDA tensor of the given dtype and exactly
    n elements (or None -> NULL): the library reads or writes n elements there."""
    if t is None:
        return None
    if t.dtype != dtype:
        raise ValueError(f"{what}: expected {dtype}, got {t.dtype}")
    if t.numel() != n:
        raise ValueError(f"{what}: expected {n} elements, got {t.numel()}")
    return _ptr(t, dtype.itemsize)


def _fptr(t, n, what):
    """Device pointer of a contiguous float32 CUDA tensor of exactly n elements (or None)."""
    import torch
    return _tptr(t, torch.float32, n, what)


def _hptr(a, n, what):
    """Address of a C-contiguous float32 host array of exactly n elements (or None)."""
    if a is None:
        return None
    if a.dtype != np.float32 or not a.flags.c_contiguous:
        raise ValueError(f"{what}: expected a C-contiguous float32 array")
    if a.size != n:
        raise ValueError(f"{what}: expected {n} elements, got {a.size}")
    return ctypes.c_void_p(a.ctypes.data)


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


@dataclass
class Params:
    """Mirror of ``sf_params``; ``None`` fields take the library defaults."""
    fx: float | None = None
    fy: float | None = None
    cx: float | None = None
    cy: float | None = None
    iters: list | None = None
    max_flow: float | None = None
    smooth: list | None = None
    gamma: tuple | None = None
    lambda_ref: float | None = None
    flags: int | None = None
    nf_max: int | None = None
    update_mode: int | None = None
    solve_tile: int | None = None

    def to_c(self, H, W, levels) -> CParams:
        c = CParams()
        _check(lib().sf_params_default(ctypes.byref(c), H, W, levels), "sf_params_default")
        for name in ("fx", "fy", "cx", "cy", "max_flow", "lambda_ref", "flags", "nf_max", "update_mode", "solve_tile"):
            v = getattr(self, name)
            if v is not None:
                setattr(c, name, v)
        if self.iters is not None:
            for k, v in enumerate(self.iters[:MAX_LEVELS]):
                c.iters[k] = int(v)
        if self.smooth is not None:
            for k, v in enumerate(self.smooth[:MAX_LEVELS]):
                c.smooth_iters[k] = int(v)
        if self.gamma is not None:
            for k, v in enumerate(self.gamma):
                c.gamma[k] = float(v)
        return c


class Filter:
    """One filter context (``sf_create`` .. ``sf_destroy``) on the current CUDA device."""

    def __init__(self, H: int, W: int, levels: int, params: Params | None = None):
        self.H, self.W, self.levels = H, W, levels
        self.params = (params or Params()).to_c(H, W, levels)
        h = ctypes.c_void_p()
        _check(lib().sf_create(H, W, levels, ctypes.byref(self.params), ctypes.byref(h)), "sf_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().sf_destroy(self._h)
            self._h = ctypes.c_void_p()

    __del__ = close

    def reset(self):
        _check(lib().sf_reset(self._h), "sf_reset")

    def step(self, image, rng, dt, flow_out=None, invdepth_out=None, stream=None):
        """Asynchronous frame on CUDA tensors; returns the status code (>= 0)."""
        n = self.H * self.W
        return _check(lib().sf_step(self._h, _fptr(image, n, "image"), _fptr(rng, n, "range"), float(dt),
                                    _fptr(flow_out, 3 * n, "flow_out"), _fptr(invdepth_out, n, "invdepth_out"),
                                    _stream(stream)), "sf_step")

    def step_host(self, image: np.ndarray, rng: np.ndarray, dt, flow_out: np.ndarray | None = None,
                  invdepth_out: np.ndarray | None = None, stream=None):
        """Frame on host float32 arrays (copies included); waits for completion."""
        n = self.H * self.W
        return _check(lib().sf_step_host(self._h, _hptr(image, n, "image"), _hptr(rng, n, "range"), float(dt),
                                         _hptr(flow_out, 3 * n, "flow_out"), _hptr(invdepth_out, n, "invdepth_out"),
                                         _stream(stream)), "sf_step_host")

    def submit_host(self, image: np.ndarray, rng: np.ndarray, dt, flow_out: np.ndarray | None = None,
                    invdepth_out: np.ndarray | None = None, stream=None) -> int:
        """Pipelined frame on host float32 arrays: enqueues the copies and the
        step and returns the frame's ticket at once.  The arrays must stay
        alive and unchanged (outputs unread) until ``wait_host(ticket)``."""
        n = self.H * self.W
        t = ctypes.c_longlong(-1)
        _check(lib().sf_submit_host(self._h, _hptr(image, n, "image"), _hptr(rng, n, "range"), float(dt),
                                    _hptr(flow_out, 3 * n, "flow_out"), _hptr(invdepth_out, n, "invdepth_out"),
                                    _stream(stream), ctypes.byref(t)), "sf_submit_host")
        return t.value

    def wait_host(self, ticket: int = -1):
        """Wait for frame ``ticket``'s outputs (-1: every submitted frame)."""
        _check(lib().sf_wait_host(self._h, int(ticket)), "sf_wait_host")

    def kernels_per_step(self) -> int:
        return _check(lib().sf_kernels_per_step(self._h), "sf_kernels_per_step")

    def nf_max(self) -> int:
        """Sub-iterations fused per propagation launch (set, or chosen by AUTOTUNE)."""
        return _check(lib().sf_nf_max(self._h), "sf_nf_max")

    def update_mode(self) -> int:
        """1: smoothing + reconstruction cascade; 2: all smoothing, then reconstruction."""
        return _check(lib().sf_update_mode(self._h), "sf_update_mode")

    def solve_tile(self) -> int:
        """Edge of the solve launch's pixel tiles (16 or 32; set, default or AUTOTUNE)."""
        return _check(lib().sf_solve_tile(self._h), "sf_solve_tile")

    def set_surrogate(self, net):
        """Predict the top level with a trained Surrogate (None: the plain propagation)."""
        _check(lib().sf_set_surrogate(self._h, None if net is None else net._h), "sf_set_surrogate")
        self._surrogate = net     # kept alive while attached

    def set_surrogate_threshold(self, threshold_px):
        """Fallback threshold of the attached surrogate (px/frame; inf: never)."""
        _check(lib().sf_set_surrogate_threshold(self._h, ctypes.c_float(threshold_px)), "sf_set_surrogate_threshold")

    def surrogate_stats(self):
        """(last frame's residual against one plain step in px/frame, frames that fell back)."""
        r, c = ctypes.c_float(), ctypes.c_int()
        _check(lib().sf_surrogate_stats(self._h, ctypes.byref(r), ctypes.byref(c)), "sf_surrogate_stats")
        return r.value, c.value

    def set_motion(self, omega=None, accel=None, stream=None):
        """Angular velocity (rad/s) and linear acceleration (m/s^2) for IMU steps."""
        om = None if omega is None else (ctypes.c_float * 3)(*[float(x) for x in omega])
        ac = None if accel is None else (ctypes.c_float * 3)(*[float(x) for x in accel])
        _check(lib().sf_set_motion(self._h, om, ac, _stream(stream)), "sf_set_motion")

    def profile(self, enable: bool):
        _check(lib().sf_profile(self._h, int(bool(enable))), "sf_profile")

    def profile_read(self):
        """(summed ms, launch count) per launch slot since the last read."""
        n = 16
        ms = (ctypes.c_float * n)(); cnt = (ctypes.c_int * n)()
        slots = _check(lib().sf_profile_read(self._h, ms, cnt, n), "sf_profile_read")
        return [(ms[k], cnt[k]) for k in range(min(slots, n))]

    def status(self) -> int:
        """OK, WARN_CFL or ENONFINITE recorded since the last call; raises on a failed call."""
        code = lib().sf_status(self._h)
        if code not in (OK, WARN_CFL, ENONFINITE):
            raise SFError(code, "sf_status")
        return code

    def level_shape(self, h):
        return self.H >> h, self.W >> h

    def get_state(self, h, stream=None):
        """Level h (0-based) state as an [8, H_h, W_h] CUDA tensor and dt_prev."""
        import torch
        Hh, Wh = self.level_shape(h)
        dst = torch.empty((8, Hh, Wh), dtype=torch.float32, device="cuda")
        dtp = ctypes.c_float()
        _check(lib().sf_get_state(self._h, h, _ptr(dst), ctypes.byref(dtp), _stream(stream)), "sf_get_state")
        return dst, dtp.value

    def set_state(self, h, planes, dt_prev, stream=None):
        Hh, Wh = self.level_shape(h)
        _check(lib().sf_set_state(self._h, h, _fptr(planes.contiguous(), 8 * Hh * Wh, "planes"), float(dt_prev),
                                  _stream(stream)), "sf_set_state")


def grid(H, W, fx, fy, cx, cy) -> CGrid:
    return CGrid(int(H), int(W), float(fx), float(fy), float(cx), float(cy))


def propagate(g: CGrid, N, s0_in, s0_out, s1_in=None, s1_out=None, flags=0, wscale=1.0, status=None,
              stream=None):
    """Stage entry point ``sf_propagate`` on [H, W, 4] float32 CUDA tensors."""
    n = 4 * g.H * g.W
    return _check(lib().sf_propagate(ctypes.byref(g), int(N), int(flags), float(wscale), _fptr(s0_in, n, "s0_in"),
                                     _fptr(s1_in, n, "s1_in"), _fptr(s0_out, n, "s0_out"), _fptr(s1_out, n, "s1_out"),
                                     _ptr(status), _stream(stream)), "sf_propagate")


def propagate_imu(g: CGrid, N, imu, s0_in, s0_out, s1_in=None, s1_out=None, flags=0, wscale=1.0, status=None,
                  stream=None):
    """``sf_propagate_imu``: imu = (Omega, a) in frame units, six numbers."""
    m = (ctypes.c_float * 6)(*[float(x) for x in np.asarray(imu, dtype=np.float64).reshape(6)])
    n = 4 * g.H * g.W
    return _check(lib().sf_propagate_imu(ctypes.byref(g), int(N), int(flags), float(wscale), m,
                                         _fptr(s0_in, n, "s0_in"), _fptr(s1_in, n, "s1_in"),
                                         _fptr(s0_out, n, "s0_out"), _fptr(s1_out, n, "s1_out"), _ptr(status),
                                         _stream(stream)), "sf_propagate_imu")


def propagate_noalloc(g: CGrid, N, s0_in, s0_out, s1_in=None, s1_out=None, flags=0, wscale=1.0, status=None,
                      stream=None):
    """``sf_propagate_noalloc``: sf_propagate without allocating (frames up to 1024 x 1024 pixels)."""
    n = 4 * g.H * g.W
    return _check(lib().sf_propagate_noalloc(ctypes.byref(g), int(N), int(flags), float(wscale),
                                             _fptr(s0_in, n, "s0_in"), _fptr(s1_in, n, "s1_in"),
                                             _fptr(s0_out, n, "s0_out"), _fptr(s1_out, n, "s1_out"), _ptr(status),
                                             _stream(stream)), "sf_propagate_noalloc")


def update(g: CGrid, level, top, S, init, gamma, lambda_ref, image, rng, s0_new, s1_new, s0_cur=None, s1_cur=None,
           p0=None, p1=None, diag=None, stream=None):
    """Stage entry point ``sf_update``; image/rng are the level-1 [H1, W1] inputs."""
    gm = (ctypes.c_float * 5)(*gamma)
    H1, W1 = image.shape
    n1, n = H1 * W1, 4 * g.H * g.W
    return _check(lib().sf_update(ctypes.byref(g), int(level), int(top), int(S), int(init), gm, float(lambda_ref),
                                  _fptr(image, n1, "image"), _fptr(rng, n1, "range"), H1, W1,
                                  _fptr(s0_cur, n, "s0_cur"), _fptr(s1_cur, n, "s1_cur"), _fptr(p0, n, "p0"),
                                  _fptr(p1, n, "p1"), _fptr(s0_new, n, "s0_new"), _fptr(s1_new, n, "s1_new"),
                                  _fptr(diag, 3 * n, "diag"), _stream(stream)), "sf_update")


def reconstruct(grids, s0, s1, dt, flow_out=None, invdepth_out=None, check_finite=False, status=None, stream=None):
    """Stage entry point ``sf_reconstruct`` over per-level [H, W, 4] tensors."""
    L = len(grids)
    ga = (CGrid * L)(*grids)
    p0 = (ctypes.c_void_p * L)(*[_fptr(t, 4 * gr.H * gr.W, "s0").value for t, gr in zip(s0, grids)])
    p1 = (ctypes.c_void_p * L)(*[_fptr(t, 4 * gr.H * gr.W, "s1").value for t, gr in zip(s1, grids)])
    n = grids[0].H * grids[0].W
    return _check(lib().sf_reconstruct(L, ga, p0, p1, float(dt), _fptr(flow_out, 3 * n, "flow_out"),
                                       _fptr(invdepth_out, n, "invdepth_out"), int(bool(check_finite)), _ptr(status),
                                       _stream(stream)), "sf_reconstruct")


def remap_pinhole(dst: CGrid, R, cam, image, out_image, rng=None, out_range=None, stream=None):
    """``sf_remap_pinhole``: a pinhole frame (device [Hs, Ws]) onto the grid ``dst``."""
    Rm = (ctypes.c_float * 9)(*[float(x) for x in np.asarray(R, dtype=np.float64).reshape(9)])
    K = (ctypes.c_float * 4)(*[float(x) for x in cam])
    Hs, Ws = image.shape
    n, nd = Hs * Ws, dst.H * dst.W
    return _check(lib().sf_remap_pinhole(ctypes.byref(dst), Rm, Hs, Ws, K, _fptr(image, n, "image"),
                                         _fptr(rng, n, "rng"), _fptr(out_image, nd, "out_image"),
                                         _fptr(out_range, nd, "out_range"), _stream(stream)), "sf_remap_pinhole")


def remap_equirect(dst: CGrid, R, image, out_image, rng=None, out_range=None, stream=None):
    """``sf_remap_equirect``: an equirectangular panorama (device [Hs, Ws]) onto the grid ``dst``."""
    Rm = (ctypes.c_float * 9)(*[float(x) for x in np.asarray(R, dtype=np.float64).reshape(9)])
    Hs, Ws = image.shape
    n, nd = Hs * Ws, dst.H * dst.W
    return _check(lib().sf_remap_equirect(ctypes.byref(dst), Rm, Hs, Ws, _fptr(image, n, "image"),
                                          _fptr(rng, n, "rng"), _fptr(out_image, nd, "out_image"),
                                          _fptr(out_range, nd, "out_range"), _stream(stream)), "sf_remap_equirect")


def conv3x3(x, w, bias=None, relu=False, y=None, y32=None, status=None, stream=None):
    """``sf_conv3x3``: x [N, H, W, Cin] and w [9, Cout, Cin] bfloat16 CUDA tensors; writes y
    (bfloat16) and/or y32 (float32), [N, H, W, Cout]."""
    import torch
    N, H, W, Cin = x.shape
    if w.dim() != 3 or w.shape[0] != 9 or w.shape[2] != Cin:
        raise ValueError(f"w: expected [9, Cout, {Cin}], got {list(w.shape)}")
    Cout = w.shape[1]
    bf, f32 = torch.bfloat16, torch.float32
    m = N * H * W * Cout
    return _check(lib().sf_conv3x3(N, H, W, Cin, Cout, _tptr(x, bf, x.numel(), "x"), _tptr(w, bf, w.numel(), "w"),
                                   _tptr(bias, f32, Cout, "bias"), int(bool(relu)), _tptr(y, bf, m, "y"),
                                   _tptr(y32, f32, m, "y32"), _tptr(status, torch.int32, 1, "status"),
                                   _stream(stream)), "sf_conv3x3")


def set_trace(enable):
    """``sf_set_trace``: NVTX ranges around every frame and stage launch (off by default)."""
    return _check(lib().sf_set_trace(int(bool(enable))), "sf_set_trace")


def conv3x3_wgrad(x, dy, dw, db, stream=None):
    """``sf_conv3x3_wgrad``: x [N, H, W, Cin] and dy [N, H, W, Cout] bfloat16 CUDA tensors;
    overwrites dw [9, Cout, Cin] and db [Cout] (float32)."""
    import torch
    N, H, W, Cin = x.shape
    if dy.dim() != 4 or tuple(dy.shape[:3]) != (N, H, W):
        raise ValueError(f"dy: expected [{N}, {H}, {W}, Cout], got {list(dy.shape)}")
    Cout = dy.shape[3]
    bf, f32 = torch.bfloat16, torch.float32
    return _check(lib().sf_conv3x3_wgrad(N, H, W, Cin, Cout, _tptr(x, bf, x.numel(), "x"),
                                         _tptr(dy, bf, dy.numel(), "dy"), _tptr(dw, f32, 9 * Cout * Cin, "dw"),
                                         _tptr(db, f32, Cout, "db"), _stream(stream)), "sf_conv3x3_wgrad")


class Surrogate:
    """The learned propagation surrogate (``sf_surrogate_*``)."""

    LAYERS = ((16, 32), (32, 32), (32, 32), (32, 16))

    def __init__(self, seed=0):
        h = ctypes.c_void_p()
        _check(lib().sf_surrogate_create(int(seed), ctypes.byref(h)), "sf_surrogate_create")
        self._h = h
        self.n_params = _check(lib().sf_surrogate_num_params(h), "sf_surrogate_num_params")

    def params(self):
        out = np.empty(self.n_params, np.float32)
        _check(lib().sf_surrogate_params(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), 0),
               "sf_surrogate_params")
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.n_params
        _check(lib().sf_surrogate_params(self._h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), 1),
               "sf_surrogate_params")

    def grads(self):
        out = np.empty(self.n_params, np.float32)
        _check(lib().sf_surrogate_grads(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
               "sf_surrogate_grads")
        return out

    def forward(self, g: CGrid, s0, p0, stream=None, layered=False):
        """s0, p0: [n, H, W, 4] float32 CUDA tensors (top-level state, w in rad/frame).
        layered: the layer-by-layer form (activations through HBM) instead of the fused kernel."""
        n = s0.shape[0] if s0.dim() == 4 else 1
        fn = lib().sf_surrogate_forward_layered if layered else lib().sf_surrogate_forward
        return _check(fn(self._h, ctypes.byref(g), n, _ptr(s0), _ptr(p0), _stream(stream)),
                      "sf_surrogate_forward_layered" if layered else "sf_surrogate_forward")

    def train_step(self, g: CGrid, s0, target, lr, stream=None):
        n = s0.shape[0] if s0.dim() == 4 else 1
        loss = ctypes.c_float()
        _check(lib().sf_surrogate_train_step(self._h, ctypes.byref(g), n, _ptr(s0), _ptr(target), float(lr),
                                             ctypes.byref(loss), _stream(stream)), "sf_surrogate_train_step")
        return loss.value

    def propagate(self, g: CGrid, N, s0, p0, threshold_px, stream=None):
        """Prediction with the plain fallback; returns (residual px, used_plain)."""
        n = s0.shape[0] if s0.dim() == 4 else 1
        res = ctypes.c_float(); used = ctypes.c_int()
        _check(lib().sf_surrogate_propagate(self._h, ctypes.byref(g), n, int(N), _ptr(s0), _ptr(p0),
                                            float(threshold_px), ctypes.byref(res), ctypes.byref(used),
                                            _stream(stream)), "sf_surrogate_propagate")
        return res.value, bool(used.value)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().sf_surrogate_destroy(self._h)
            self._h = ctypes.c_void_p()

    __del__ = close


class Batch:
    """Many independent filters (``sf_batch_*``); stream s has its own device
    input/output slots, exposed as torch tensors viewing the batch's memory."""

    def __init__(self, shapes, levels, params):
        import torch
        n = len(shapes)
        Hs = (ctypes.c_int * n)(*[int(h) for h, _ in shapes])
        Ws = (ctypes.c_int * n)(*[int(w) for _, w in shapes])
        Ls = (ctypes.c_int * n)(*[int(x) for x in levels])
        ps = (CParams * n)(*[p.to_c(h, w, l) for p, (h, w), l in zip(params, shapes, levels)])
        h = ctypes.c_void_p()
        _check(lib().sf_batch_create(n, Hs, Ws, Ls, ps, ctypes.byref(h)), "sf_batch_create")
        self._h = h
        self.shapes = list(shapes)
        self.slots = []
        for s, (H, W) in enumerate(shapes):
            ptrs = [ctypes.c_void_p() for _ in range(4)]
            _check(lib().sf_batch_buffers(h, s, *[ctypes.byref(x) for x in ptrs]), "sf_batch_buffers")
            self.slots.append(tuple(_wrap(x.value, shp) for x, shp in
                                    zip(ptrs, [(H, W), (H, W), (3, H, W), (H, W)])))
        self.motion = []      # per stream: 6-float device view, Omega (rad/s) then a (m/s^2)
        for s in range(n):
            mp = ctypes.c_void_p()
            _check(lib().sf_batch_motion(h, s, ctypes.byref(mp)), "sf_batch_motion")
            self.motion.append(_wrap(mp.value, (6,)))

    def step(self, dt, stream=None):
        return _check(lib().sf_batch_step(self._h, float(dt), _stream(stream)), "sf_batch_step")

    def set_surrogate(self, net):
        _check(lib().sf_batch_set_surrogate(self._h, None if net is None else net._h), "sf_batch_set_surrogate")
        self._surrogate = net

    def set_surrogate_threshold(self, threshold_px, stream=-1):
        """Fallback threshold (px/frame; inf: never) of batch stream `stream` (-1: all)."""
        _check(lib().sf_batch_set_surrogate_threshold(self._h, int(stream), ctypes.c_float(threshold_px)),
               "sf_batch_set_surrogate_threshold")

    def surrogate_stats(self):
        """Per stream: (last frame's residual in px/frame, frames that fell back) as numpy arrays."""
        n = len(self.shapes)
        r, c = (ctypes.c_float * n)(), (ctypes.c_int * n)()
        _check(lib().sf_batch_surrogate_stats(self._h, r, c, n), "sf_batch_surrogate_stats")
        return np.array(r[:], dtype=np.float64), np.array(c[:], dtype=np.int64)

    def status(self):
        code = lib().sf_batch_status(self._h)
        if code not in (OK, WARN_CFL, ENONFINITE):
            raise SFError(code, "sf_batch_status")
        return code

    def launches_per_step(self):
        return _check(lib().sf_batch_launches_per_step(self._h), "sf_batch_launches_per_step")

    def nf_max(self) -> int:
        return _check(lib().sf_batch_nf_max(self._h), "sf_batch_nf_max")

    def update_mode(self) -> int:
        return _check(lib().sf_batch_update_mode(self._h), "sf_batch_update_mode")

    def solve_tile(self) -> int:
        return _check(lib().sf_batch_solve_tile(self._h), "sf_batch_solve_tile")

    def profile(self, enable: bool):
        _check(lib().sf_batch_profile(self._h, int(bool(enable))), "sf_batch_profile")

    def profile_read(self):
        n = 16
        ms = (ctypes.c_float * n)(); cnt = (ctypes.c_int * n)()
        slots = _check(lib().sf_batch_profile_read(self._h, ms, cnt, n), "sf_batch_profile_read")
        return [(ms[k], cnt[k]) for k in range(min(slots, n))]

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().sf_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    __del__ = close


def _wrap(ptr, shape):
    """A float32 CUDA tensor viewing library-owned device memory (no copy)."""
    import torch
    n = int(np.prod(shape))

    class _Iface:
        __cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<f4", "data": (int(ptr), False),
                                    "version": 3, "strides": None}
    return torch.as_tensor(_Iface(), device="cuda")
