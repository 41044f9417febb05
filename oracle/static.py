"""Closed-form box-to-box integrals of 1/r (the quasi-static kernel).

Test infrastructure (see ``oracle/__init__``).

B(D) = int_{box n} int_{box m} dV dV0 / |r - r0| for a field box n and a source
box m with equal lateral sizes hx, hy and z-extents [zf1, zf2], [zs1, zs2]; D is
the lateral offset (x_n - x_m, y_n - y_m).  Its second derivatives with respect
to the offsets are what the static part of the Galerkin coefficients needs:

  d2B/dDx2 = int_n d2/dx2 int_m 1/r  (and y, z, xy, xz, yz likewise),

with the z-derivative acting on the field box position.  They are sums over the
corners of the Minkowski difference of the boxes of 4-fold antiderivatives of 1/r:

  P(x; y, z):  d^2/dy^2 d^2/dz^2 P = 1/r     (parallel faces)
  N(x, z; y):  d/dx d/dz d^2/dy^2 N = 1/r    (perpendicular faces)

Both were derived by repeated integration of the textbook two-fold antiderivative
y ln(z+r) + z ln(y+r) - x atan(yz/(xr)) and checked by differentiation; terms that
the corner sums annihilate (polynomials of degree <= 1 in a stencil variable)
were dropped.  The corner stencils are: lateral (1, -2, 1) at D - h, D, D + h;
vertical (1, -1, -1, 1) at zf2 - zs1, zf2 - zs2, zf1 - zs1, zf1 - zs2.

Pins: direct numerical quadrature of the same integrals, including touching and
overlapping boxes (tests/test_oracle_static.py), and the spectral identity
int_0^inf K_J(lam) e^{-lam a} dlam = tent-weighted lateral integral of 1/r.
"""
from __future__ import annotations

import numpy as np


def _xlog(m, v, r, o2):
    """m * ln(v + r) with r = sqrt(v^2 + o2); m vanishes wherever v + r does."""
    with np.errstate(divide="ignore", invalid="ignore"):
        pos = v >= 0
        lg = np.where(pos, np.log(np.where(pos, v + r, 1.0)),
                      np.log(np.where(o2 > 0, o2, 1.0)) - np.log(np.where(pos, 1.0, r - v)))
        out = m * lg
    return np.where(m == 0, 0.0, out)


def _xatan(m, num, den):
    """m * atan(num / den); m vanishes wherever den does."""
    with np.errstate(divide="ignore", invalid="ignore"):
        out = m * np.arctan(num / np.where(den == 0, 1.0, den))
    return np.where(den == 0, 0.0, out)


def P(x, y, z):
    """d^2/dy^2 d^2/dz^2 P(x; y, z) = 1/sqrt(x^2+y^2+z^2)."""
    x, y, z = np.broadcast_arrays(*(np.asarray(a, dtype=np.float64) for a in (x, y, z)))
    r = np.sqrt(x * x + y * y + z * z)
    x2, y2, z2 = x * x, y * y, z * z
    out = (-0.5 * _xlog(x2 * y, y, r, x2 + z2)
           - 0.5 * _xlog(x2 * z, z, r, x2 + y2)
           + x2 * r / 3.0
           - _xatan(x * y * z, y * z, x * r)
           + 0.5 * _xlog(y2 * z, z, r, x2 + y2)
           - y2 * r / 6.0
           + 0.5 * _xlog(y * z2, y, r, x2 + z2)
           - z2 * r / 6.0)
    return out


def N(x, z, y):
    """d/dx d/dz d^2/dy^2 N(x, z; y) = 1/sqrt(x^2+y^2+z^2)."""
    x, y, z = np.broadcast_arrays(*(np.asarray(a, dtype=np.float64) for a in (x, y, z)))
    r = np.sqrt(x * x + y * y + z * z)
    x2, y2, z2 = x * x, y * y, z * z
    out = (-_xlog(x2 * x, z, r, x2 + y2) / 6.0
           - 0.5 * _xatan(x2 * y, y * z, x * r)
           + 0.5 * _xlog(x * y2, z, r, x2 + y2)
           + _xlog(x * y * z, y, r, x2 + z2)
           - x * z * r / 3.0
           - _xatan(y2 * y, x * z, y * r) / 6.0
           + 0.5 * _xlog(y2 * z, x, r, y2 + z2)
           - 0.5 * _xatan(y * z2, x * y, z * r)
           - _xlog(z2 * z, x, r, y2 + z2) / 6.0)
    return out


_LAT = ((-1.0, 1.0), (0.0, -2.0), (1.0, 1.0))   # (multiple of h, weight)


def box_d2(kind, Dx, Dy, hx, hy, zf1, zf2, zs1, zs2):
    """Second derivative of B with respect to the offsets, kind in
    {'xx','yy','zz','xy','xz','yz'}.  Dx, Dy may be arrays (broadcast)."""
    Dx = np.asarray(Dx, dtype=np.float64)
    Dy = np.asarray(Dy, dtype=np.float64)
    zst = ((zf2 - zs1, 1.0), (zf2 - zs2, -1.0), (zf1 - zs1, -1.0), (zf1 - zs2, 1.0))
    acc = np.zeros(np.broadcast(Dx, Dy).shape)
    for ax, wx in _LAT:
        X = Dx + ax * hx
        for ay, wy in _LAT:
            Y = Dy + ay * hy
            for Z, wz in zst:
                w = wx * wy * wz
                if kind == "xx":
                    v = P(X, Y, Z)
                elif kind == "yy":
                    v = P(Y, X, Z)
                elif kind == "zz":
                    v = P(Z, X, Y)
                elif kind == "xy":
                    v = N(X, Y, Z)
                elif kind == "xz":
                    v = N(X, Z, Y)
                elif kind == "yz":
                    v = N(Y, Z, X)
                else:
                    raise ValueError(kind)
                acc = acc + w * v
    return acc


def lateral_static(Dx, Dy, hx, hy, a):
    """Tent-weighted lateral integral of 1/r at vertical separation a:
    int int_{rect n} int int_{rect m} 1/sqrt(rho^2 + a^2) = sum over the 3x3 lateral
    stencil of P(a; X, Y)."""
    acc = 0.0
    for ax, wx in _LAT:
        for ay, wy in _LAT:
            acc = acc + wx * wy * P(a, Dx + ax * hx, Dy + ay * hy)
    return acc
