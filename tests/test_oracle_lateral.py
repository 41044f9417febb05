"""Pins for the lateral J0 kernels (oracle/lateral.py)."""
import numpy as np
import pytest
from scipy import integrate, special

from oracle import lateral, static

HX, HY = 50.0, 65.0


def test_zero_lambda_limit():
    k = lateral.lateral_kernels(np.array([1e-12]), 3 * HX, 2 * HY, HX, HY)
    assert abs(k["J"][0] - HX ** 2 * HY ** 2) < 1e-9 * HX ** 2 * HY ** 2
    for name in ("xx", "yy", "xy", "x", "y"):
        assert abs(k[name][0]) < 1e-6 * HX * HY


@pytest.mark.parametrize("D", [(0.0, 0.0), (50.0, 0.0), (150.0, -130.0), (-300.0, 65.0)])
@pytest.mark.parametrize("lam", [3e-3, 4e-2, 0.2])
def test_KJ_spatial_quadrature(D, lam):
    Dx, Dy = D
    f = lambda v, u: (HX - abs(u)) * (HY - abs(v)) * special.j0(lam * np.hypot(Dx + u, Dy + v))
    ref = 0.0
    for u0, u1 in ((-HX, 0.0), (0.0, HX)):
        for v0, v1 in ((-HY, 0.0), (0.0, HY)):
            ref += integrate.dblquad(f, u0, u1, v0, v1, epsabs=1e-9 * HX ** 2 * HY ** 2, epsrel=1e-11)[0]
    got = lateral.lateral_kernels(np.array([lam]), Dx, Dy, HX, HY)["J"][0]
    assert abs(got - ref) <= 1e-8 * HX ** 2 * HY ** 2, (got, ref)


@pytest.mark.parametrize("D", [(0.0, 0.0), (50.0, 65.0), (200.0, -130.0)])
def test_derivative_kernels_by_differences(D):
    Dx, Dy = D
    lam = np.array([2e-3, 1e-2, 5e-2])
    d = 1e-2
    K = lambda a, b: lateral.lateral_kernels(lam, Dx + a, Dy + b, HX, HY)["J"]
    k = lateral.lateral_kernels(lam, Dx, Dy, HX, HY)
    scale = HX * HY * HX * HY
    fd = {
        "x": (K(d, 0) - K(-d, 0)) / (2 * d),
        "y": (K(0, d) - K(0, -d)) / (2 * d),
        "xx": (K(d, 0) - 2 * K(0, 0) + K(-d, 0)) / d ** 2,
        "yy": (K(0, d) - 2 * K(0, 0) + K(0, -d)) / d ** 2,
        "xy": (K(d, d) - K(d, -d) - K(-d, d) + K(-d, -d)) / (4 * d * d),
    }
    for name, ref in fd.items():
        tol = (1e-6 if len(name) == 1 else 2e-3) * scale * lam ** len(name) + 1e-7 * scale / HX ** len(name)
        assert np.all(np.abs(k[name] - ref) <= tol), (name, k[name], ref)


@pytest.mark.parametrize("D", [(0.0, 0.0), (50.0, 0.0), (100.0, 130.0), (-250.0, 65.0)])
@pytest.mark.parametrize("a", [20.0, 75.0])
def test_sommerfeld_identity_against_closed_form(D, a):
    """int_0^inf K_J(lam) e^{-lam a} dlam = int_rect int_rect 1/sqrt(rho^2 + a^2)."""
    Dx, Dy = D
    # Gauss-Legendre on [0, 40/a] in panels (the integrand decays like e^{-lam a})
    edges = np.linspace(0.0, 40.0 / a, 161)
    xg, wg = np.polynomial.legendre.leggauss(12)
    lam = (0.5 * (edges[1:] - edges[:-1])[:, None] * xg[None, :] + 0.5 * (edges[1:] + edges[:-1])[:, None]).ravel()
    w = (0.5 * (edges[1:] - edges[:-1])[:, None] * wg[None, :]).ravel()
    kj = lateral.lateral_kernels(lam, Dx, Dy, HX, HY)["J"]
    got = np.sum(w * kj * np.exp(-lam * a))
    ref = static.lateral_static(Dx, Dy, HX, HY, a)
    assert abs(got - ref) <= 1e-10 * abs(ref), (got, ref)
