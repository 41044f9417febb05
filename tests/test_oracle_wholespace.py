"""Whole-space pin of the Galerkin coefficients (Appendix A with every layer, and the
air, given the same conductivity).

In a homogeneous space the electric Green's tensor is the textbook dyadic
G^E = i w mu0 (I + grad grad / k^2) e^{ikr} / (4 pi r), so

  B_ab = i w mu0 [ delta_ab G + (1/k^2) d2 G / dD_a dD_b ],   G(D) = int_n int_m e^{ikr}/(4 pi r),

with the derivatives on the field-cell offset.  This is computed here without the
layered-medium machinery: e^{ikr}/r = 1/r + (e^{ikr} - 1)/r; the 1/r part from the
closed-form box integrals (pinned separately against quadrature) and by adaptive
quadrature for G itself; the bounded remainder by Gauss-Legendre product rules
split at the kinks of the cell-overlap weights.  Every block (including zx and zy,
which the oracle takes from Lemma 1) and near and far offsets are compared.
"""
import numpy as np
import pytest
from scipy import integrate

from oracle import coefficients, static
from workloads import Grid, Layers

SIG = 0.05
FREQ = 300.0
OMEGA = 2 * np.pi * FREQ
MU0 = 4e-7 * np.pi
K2 = 1j * OMEGA * MU0 * SIG
K = np.sqrt(K2)            # Im k > 0: e^{ikr} decays
HX, HY = 50.0, 65.0
ZE = (0.0, 40.0, 100.0, 130.0, 200.0)
GRID = Grid(6, 5, 4, HX, HY, ZE)
LAY = Layers((0.0, 1000.0), (SIG, SIG, SIG))

XG, WG = np.polynomial.legendre.leggauss(20)


def _gl(a, b):
    return 0.5 * (b - a) * XG + 0.5 * (a + b), 0.5 * (b - a) * WG


def hfun(x, y, z):
    r = np.sqrt(x * x + y * y + z * z)
    small = r < 1e-9
    rs = np.where(small, 1.0, r)
    return np.where(small, 1j * K / (4 * np.pi), np.expm1(1j * K * rs) / (4 * np.pi * rs))


def tent_pieces(h):
    return [(-h, 0.0, lambda u: h + u), (0.0, h, lambda u: h - u)]


def sign_pieces(h):
    return [(-h, 0.0, lambda u: -np.ones_like(u)), (0.0, h, lambda u: np.ones_like(u))]


def trap_pieces(zf1, zf2, zs1, zs2):
    ks = sorted([zf1 - zs2, zf1 - zs1, zf2 - zs2, zf2 - zs1])
    T = lambda w: np.maximum(0.0, np.minimum(zf2, zs2 + w) - np.maximum(zf1, zs1 + w))
    return [(a, b, T) for a, b in zip(ks[:-1], ks[1:]) if b > a]


def zshift_pieces(zf1, zf2, zs1, zs2):
    return [(zf2 - zs2, zf2 - zs1, lambda w: np.ones_like(w)), (zf1 - zs2, zf1 - zs1, lambda w: -np.ones_like(w))]


def quad3(f, px, py, pz, cx=0.0, cy=0.0, cz=0.0):
    """sum over pieces of int wx(u) wy(v) wz(w) f(cx+u, cy+v, cz+w); pieces split at 0 shift."""
    tot = 0.0
    for (a0, a1, wa) in px:
        for (b0, b1, wb) in py:
            for (c0, c1, wc) in pz:
                u, wu = _gl(a0, a1)
                v, wv = _gl(b0, b1)
                w, ww = _gl(c0, c1)
                U, V, Wz = np.meshgrid(u, v, w, indexing="ij")
                wt = (wu * wa(u))[:, None, None] * (wv * wb(v))[None, :, None] * (ww * wc(w))[None, None, :]
                tot += np.sum(wt * f(cx + U, cy + V, cz + Wz))
    return tot


def point_pieces(x):
    """A 'piece' that evaluates at a single coordinate (for stencils)."""
    return x


def quad2_at(f, px, py, zval, cx, cy):
    tot = 0.0
    for (a0, a1, wa) in px:
        for (b0, b1, wb) in py:
            u, wu = _gl(a0, a1)
            v, wv = _gl(b0, b1)
            U, V = np.meshgrid(u, v, indexing="ij")
            tot += np.sum((wu * wa(u))[:, None] * (wv * wb(v))[None, :] * f(cx + U, cy + V, zval))
    return tot


def d2_h(kind, Dx, Dy, zf1, zf2, zs1, zs2):
    """Second offset derivative of int_n int_m h(r - r0)."""
    trap = trap_pieces(zf1, zf2, zs1, zs2)
    zsh = zshift_pieces(zf1, zf2, zs1, zs2)
    lat = ((-1, 1.0), (0, -2.0), (1, 1.0))
    if kind == "xx":
        return sum(wx * quad2_at(lambda y, z, x: hfun(x, y, z), tent_pieces(HY), trap, Dx + ax * HX, Dy, 0.0)
                   for ax, wx in lat)
    if kind == "yy":
        return sum(wy * quad2_at(lambda x, z, y: hfun(x, y, z), tent_pieces(HX), trap, Dy + ay * HY, Dx, 0.0)
                   for ay, wy in lat)
    if kind == "zz":
        zst = ((zf2 - zs1, 1.0), (zf2 - zs2, -1.0), (zf1 - zs1, -1.0), (zf1 - zs2, 1.0))
        return sum(wz * quad2_at(hfun, tent_pieces(HX), tent_pieces(HY), Z, Dx, Dy) for Z, wz in zst)
    if kind == "xy":
        return quad3(hfun, sign_pieces(HX), sign_pieces(HY), trap, Dx, Dy, 0.0)
    if kind == "xz":
        return quad3(hfun, sign_pieces(HX), tent_pieces(HY), zsh, Dx, Dy, 0.0)
    if kind == "yz":
        return quad3(hfun, tent_pieces(HX), sign_pieces(HY), zsh, Dx, Dy, 0.0)
    raise ValueError(kind)


def G0_static(Dx, Dy, zf1, zf2, zs1, zs2):
    """int_n int_m 1/r by adaptive quadrature (inner z-integral in closed form)."""
    ks = sorted([zf1 - zs2, zf1 - zs1, zf2 - zs2, zf2 - zs1])
    T = lambda w: max(0.0, min(zf2, zs2 + w) - max(zf1, zs1 + w))
    pcs = []
    for a, b in zip(ks[:-1], ks[1:]):
        if b > a:
            be = (T(b) - T(a)) / (b - a)
            pcs.append((a, b, T(a) - be * a, be))

    def inner(rho):
        rho = max(rho, 1e-300)
        tot = 0.0
        for a, b, al, be in pcs:
            F = lambda t: al * np.arcsinh(t / rho) + be * np.sqrt(rho * rho + t * t)
            tot += F(b) - F(a)
        return tot
    tot = 0.0
    for u0, u1, su in ((-HX, 0.0, 1.0), (0.0, HX, -1.0)):
        for v0, v1, sv in ((-HY, 0.0, 1.0), (0.0, HY, -1.0)):
            opts = [dict(limit=200, epsrel=1e-11), dict(limit=200, epsrel=1e-11)]
            if u0 < -Dx < u1:
                opts[1]["points"] = [-Dx]
            if v0 < -Dy < v1:
                opts[0]["points"] = [-Dy]
            tot += integrate.nquad(lambda v, u: (HX + su * u) * (HY + sv * v) * inner(np.hypot(Dx + u, Dy + v)),
                                   [(v0, v1), (u0, u1)], opts=opts)[0]
    return tot


def brute_block(i, j, a, b):
    Dx, Dy = j * HX, i * HY
    zf1, zf2, zs1, zs2 = ZE[a], ZE[a + 1], ZE[b], ZE[b + 1]
    G = G0_static(Dx, Dy, zf1, zf2, zs1, zs2) / (4 * np.pi) + quad3(
        hfun, tent_pieces(HX), tent_pieces(HY), trap_pieces(zf1, zf2, zs1, zs2), Dx, Dy, 0.0)
    d2 = {kd: static.box_d2(kd, Dx, Dy, HX, HY, zf1, zf2, zs1, zs2) / (4 * np.pi)
          + d2_h(kd, Dx, Dy, zf1, zf2, zs1, zs2) for kd in ("xx", "yy", "zz", "xy", "xz", "yz")}
    iwm = 1j * OMEGA * MU0
    B = np.empty((3, 3), dtype=np.complex128)
    B[0, 0] = iwm * (G + d2["xx"] / K2)
    B[1, 1] = iwm * (G + d2["yy"] / K2)
    B[2, 2] = iwm * (G + d2["zz"] / K2)
    B[0, 1] = B[1, 0] = iwm * d2["xy"] / K2
    B[0, 2] = B[2, 0] = iwm * d2["xz"] / K2
    B[1, 2] = B[2, 1] = iwm * d2["yz"] / K2
    return B


@pytest.fixture(scope="module")
def oracle_blocks():
    cache = {}

    def get(i, j):
        if (i, j) not in cache:
            cache[(i, j)] = coefficients.full_block(coefficients.offset_blocks(GRID, LAY, FREQ, i, j))
        return cache[(i, j)]
    return get


@pytest.mark.parametrize("ij", [(0, 0), (0, 1), (1, 1), (1, 2), (-3, 2), (2, -4)])
@pytest.mark.parametrize("ab", [(0, 0), (1, 2), (2, 1), (0, 3), (3, 3)])
def test_whole_space_blocks(oracle_blocks, ij, ab):
    i, j = ij
    a, b = ab
    nz = GRID.nz
    full = oracle_blocks(i, j)
    got = full[[a, nz + a, 2 * nz + a]][:, [b, nz + b, 2 * nz + b]]
    ref = brute_block(i, j, a, b)
    scale = np.max(np.abs(ref))
    err = np.abs(got - ref)
    assert np.all(err <= 2e-8 * scale), (ij, ab, got, ref, err / scale)
