"""Pins for the closed-form box integrals of 1/r (oracle/static.py).

Each second derivative of B is recomputed independently: the innermost integral
of 1/r against a piecewise-linear weight is done with the elementary primitive
(a asinh(t/rho) + b sqrt(rho^2 + t^2)); the remaining one or two dimensions by
adaptive quadrature (scipy).  Configurations include separated, touching
(shared face, edge, corner) and coincident boxes.
"""
import numpy as np
import pytest
from scipy import integrate

from oracle import static


def _lin_int(alpha, beta, c, rho, w0, w1):
    """int_{w0}^{w1} (alpha + beta w) / sqrt(rho^2 + (c + w)^2) dw."""
    rho = max(rho, 1e-300)
    A = alpha - beta * c

    def F(w):
        t = c + w
        return A * np.arcsinh(t / rho) + beta * np.sqrt(rho * rho + t * t)
    return F(w1) - F(w0)


def _pieces_tent(h):
    return [(-h, 0.0, h, 1.0), (0.0, h, h, -1.0)]          # (w0, w1, alpha, beta)


def _pieces_sign(h):
    return [(-h, 0.0, -1.0, 0.0), (0.0, h, 1.0, 0.0)]


def _pieces_trap(zf1, zf2, zs1, zs2):
    ks = sorted([zf1 - zs2, zf1 - zs1, zf2 - zs2, zf2 - zs1])
    T = lambda w: max(0.0, min(zf2, zs2 + w) - max(zf1, zs1 + w))
    out = []
    for a, b in zip(ks[:-1], ks[1:]):
        if b - a <= 0:
            continue
        ta, tb = T(a), T(b)
        beta = (tb - ta) / (b - a)
        out.append((a, b, ta - beta * a, beta))
    return out


def _pieces_zshift(zf1, zf2, zs1, zs2):
    """d/dDz of the z double integral = [int_s f(zf2 - z0) - int_s f(zf1 - z0)] dz0,
    written as weights over w = z - z0: +1 on [zf2 - zs2, zf2 - zs1], -1 on [zf1 - zs2, zf1 - zs1]."""
    return [(zf2 - zs2, zf2 - zs1, 1.0, 0.0), (zf1 - zs2, zf1 - zs1, -1.0, 0.0)]


def _inner(pieces, c, rho):
    return sum(_lin_int(al, be, c, rho, w0, w1) for (w0, w1, al, be) in pieces)


def _outer1(fun, pieces, extra_pts=()):
    tot = 0.0
    for (w0, w1, al, be) in pieces:
        pts = [p for p in extra_pts if w0 < p < w1]
        tot += integrate.quad(lambda v: (al + be * v) * fun(v), w0, w1, points=pts or None,
                              epsabs=1e-13, epsrel=1e-12, limit=400)[0]
    return tot


def _outer2(fun, pu, pv, pts_u=(), pts_v=()):
    tot = 0.0
    for (u0, u1, au, bu) in pu:
        for (v0, v1, av, bv) in pv:
            opts = []
            for pts, lo, hi in ((pts_u, u0, u1), (pts_v, v0, v1)):
                o = dict(limit=200, epsabs=1e-12, epsrel=1e-10)
                inside = [p for p in pts if lo < p < hi]
                if inside:
                    o["points"] = inside
                opts.append(o)
            tot += integrate.nquad(lambda v, u: (au + bu * u) * (av + bv * v) * fun(u, v),
                                   [(v0, v1), (u0, u1)], opts=opts[::-1])[0]
    return tot


def brute(kind, Dx, Dy, hx, hy, zf1, zf2, zs1, zs2):
    trap = _pieces_trap(zf1, zf2, zs1, zs2)
    zsh = _pieces_zshift(zf1, zf2, zs1, zs2)
    if kind in ("xx", "yy"):
        if kind == "yy":
            Dx, Dy, hx, hy = Dy, Dx, hy, hx
        tot = 0.0
        for ax, wx in ((-1, 1.0), (0, -2.0), (1, 1.0)):
            X = Dx + ax * hx
            f = lambda v: _inner(trap, 0.0, np.hypot(X, Dy + v))
            tot += wx * _outer1(f, _pieces_tent(hy), extra_pts=(-Dy,))
        return tot
    if kind == "zz":
        tot = 0.0
        for Z, wz in ((zf2 - zs1, 1.0), (zf2 - zs2, -1.0), (zf1 - zs1, -1.0), (zf1 - zs2, 1.0)):
            f = lambda v: _inner(_pieces_tent(hx), Dx, np.hypot(Z, Dy + v))
            tot += wz * _outer1(f, _pieces_tent(hy), extra_pts=(-Dy,))
        return tot
    if kind == "xy":
        f = lambda u, v: _inner(trap, 0.0, np.hypot(Dx + u, Dy + v))
        return _outer2(f, _pieces_sign(hx), _pieces_sign(hy), (-Dx,), (-Dy,))
    if kind in ("xz", "yz"):
        if kind == "yz":
            Dx, Dy, hx, hy = Dy, Dx, hy, hx
        f = lambda u, v: _inner(zsh, 0.0, np.hypot(Dx + u, Dy + v))
        return _outer2(f, _pieces_sign(hx), _pieces_tent(hy), (-Dx,), (-Dy,))
    raise ValueError(kind)


CONFIGS = [
    # Dx, Dy, hx, hy, zf1, zf2, zs1, zs2
    (3.0, 2.0, 1.0, 1.3, 0.0, 1.0, 2.0, 2.7),      # separated
    (1.0, 0.0, 1.0, 1.3, 0.0, 1.0, 0.0, 1.0),      # shared x-face, same z
    (0.0, 0.0, 1.0, 1.3, 0.0, 1.0, 0.0, 1.0),      # coincident
    (0.0, 0.0, 1.0, 1.3, 0.0, 1.0, 1.0, 1.6),      # shared z-face
    (1.0, 1.3, 1.0, 1.3, 0.0, 1.0, 1.0, 2.5),      # shared corner
    (-2.0, 1.3, 1.0, 1.3, 0.5, 1.0, -1.0, 0.5),    # negative offset, touching in z
]


@pytest.mark.parametrize("cfg", CONFIGS)
@pytest.mark.parametrize("kind", ["xx", "yy", "zz", "xy", "xz", "yz"])
def test_box_second_derivatives(kind, cfg):
    got = static.box_d2(kind, *cfg)
    ref = brute(kind, *cfg)
    assert abs(got - ref) <= 2e-8 * max(1.0, abs(ref)), (kind, cfg, got, ref)


def test_antiderivatives_by_differences():
    rng = np.random.default_rng(3)
    for _ in range(20):
        x, y, z = rng.uniform(-2, 2, 3)
        h = 1e-2
        # P: fourth mixed difference in y, z
        d = 0.0
        for a, wa in ((-1, 1), (0, -2), (1, 1)):
            for b, wb in ((-1, 1), (0, -2), (1, 1)):
                d += wa * wb * static.P(x, y + a * h, z + b * h)
        d /= h ** 4
        assert abs(d - 1 / np.sqrt(x * x + y * y + z * z)) < 2e-3 * (1 / np.sqrt(x * x + y * y + z * z))
