"""Exact-arithmetic hand stepper for the upwind prediction scheme (Sec. 4.6).

An independent, deliberately naive statement of Eqs. 53-66 over Python
``fractions.Fraction`` values, for tiny grids.  It shares no code with the C
oracle; the tests feed both the same inputs (the float64 geometry converted
exactly to rationals) and require agreement to round-off.

Readings follow the oracle's: larger-magnitude dominant speed with ties to the
minus-side neighbour (R1), row operator in the row pass (R2), replicated
borders (R13), the full source in both passes unless ``split`` (R22), and the
inertial terms once per sub-iteration after both passes when ``imu`` is given
(R23-R25).
"""
from fractions import Fraction as Fr


def _dot(a, b):
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]


def _proj(eta, v):
    d = _dot(eta, v)
    return [v[k] - eta[k] * d for k in range(3)]


def _cross(a, b):
    return [a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]]


def propagate(H, W, N, eta, b1, b2, dmu, w, rho, dw=None, Y=None, split=False, imu=None):
    """Returns (w, rho, dw, Y) after N sub-iterations; all arguments are nested
    lists [i][j] of Fractions (vectors as 3-lists); ``imu`` = (Omega, a), two
    3-lists of Fractions in frame units."""
    dt = Fr(1, N)
    sdt = dt / 2 if split else dt

    def clamp(v, hi):
        return min(max(v, 0), hi)

    for _ in range(N):
        for axis in (0, 1):
            basis = b1 if axis == 0 else b2
            speed = [[_dot(basis[i][j], _proj(eta[i][j], w[i][j])) / dmu[i][j] for j in range(W)] for i in range(H)]

            def nb(i, j, s):
                if axis == 0:
                    return i, clamp(j + s, W - 1)
                return clamp(i + s, H - 1), j

            nw = [[None] * W for _ in range(H)]
            nr = [[None] * W for _ in range(H)]
            nd = [[None] * W for _ in range(H)] if dw is not None else None
            ny = [[None] * W for _ in range(H)] if Y is not None else None
            for i in range(H):
                for j in range(W):
                    im, jm = nb(i, j, -1)
                    ip, jp = nb(i, j, +1)
                    sm, sp = speed[im][jm], speed[ip][jp]
                    s = sp if abs(sp) - abs(sm) > 0 else sm
                    src = _dot(eta[i][j], w[i][j])

                    def upd(fm, f0, fp, with_source=True):
                        D = (f0 - fm) if s > 0 else (fp - f0)
                        out = f0 - dt * s * D
                        if with_source:
                            out -= sdt * f0 * src
                        return out

                    nw[i][j] = [upd(w[im][jm][k], w[i][j][k], w[ip][jp][k]) for k in range(3)]
                    nr[i][j] = upd(rho[im][jm], rho[i][j], rho[ip][jp])
                    if dw is not None:
                        nd[i][j] = [upd(dw[im][jm][k], dw[i][j][k], dw[ip][jp][k]) for k in range(3)]
                    if Y is not None:
                        ny[i][j] = upd(Y[im][jm], Y[i][j], Y[ip][jp], with_source=False)
            w, rho, dw, Y = nw, nr, nd, ny
        if imu is not None:
            om, acc = imu
            for i in range(H):
                for j in range(W):
                    ow = _cross(om, w[i][j])
                    ooe = _cross(om, _cross(om, eta[i][j]))
                    w[i][j] = [w[i][j][k] + dt * (-2 * ow[k] - ooe[k] - rho[i][j] * acc[k]) for k in range(3)]
                    if dw is not None:
                        od = _cross(om, dw[i][j])
                        dw[i][j] = [dw[i][j][k] - dt * 2 * od[k] for k in range(3)]
    return w, rho, dw, Y


def to_fr(a):
    """numpy array -> nested lists of exact Fractions."""
    if a.ndim == 0:
        return Fr(float(a))
    return [to_fr(x) for x in a]


def to_float(x):
    if isinstance(x, list):
        return [to_float(v) for v in x]
    return float(x)
