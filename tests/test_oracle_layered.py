"""Pins for the oracle's fundamental functions and vertical integrals (Appendix B)."""
import numpy as np
import pytest
from scipy import integrate

from oracle import layered
from tests.bvp_reference import solve_U
from workloads import Layers, AIR_SIGMA

LAY = Layers((0.0, 300.0, 800.0, 1500.0), (AIR_SIGMA, 1 / 50.0, 1 / 5.0, 1 / 400.0, 1 / 20.0))
OMEGA = 2 * np.pi * 3.0


@pytest.mark.parametrize("gamma", ["1", "sigma"])
@pytest.mark.parametrize("lam", [1e-5, 3e-3, 2e-2])
@pytest.mark.parametrize("zs", [120.0, 650.0, 1700.0])
def test_U_matches_plain_bvp(gamma, lam, zs):
    """(pq_req)+(A_rs)+(UU2) equal the plain linear solve of (lmff)."""
    U_ref = solve_U(LAY, OMEGA, lam, gamma, zs)
    for z in [10.0, 120.0, 299.0, 301.0, 650.0, 799.0, 900.0, 1499.0, 1700.0, 2600.0]:
        u = layered.evaluate_U(LAY, OMEGA, lam, gamma, z, zs)[0]
        ref = U_ref(z)
        assert abs(u - ref) <= 1e-10 * abs(ref) + 1e-300, (z, u, ref)


@pytest.mark.parametrize("gamma", ["1", "sigma"])
def test_U_interface_and_jump_conditions(gamma):
    lam, zs = 4e-3, 650.0
    sig = LAY.sigma
    for m, dm in enumerate(LAY.interfaces[1:], start=1):
        up = layered.evaluate_U(LAY, OMEGA, lam, gamma, dm - 1e-9, zs)[0]
        dn = layered.evaluate_U(LAY, OMEGA, lam, gamma, dm, zs)[0]
        assert abs(up - dn) < 1e-8 * abs(dn)
        gu = 1.0 if gamma == "1" else sig[m]
        gd = 1.0 if gamma == "1" else sig[m + 1]
        du = layered.evaluate_dU(LAY, OMEGA, lam, gamma, dm - 1e-9, zs)[0] / gu
        dd = layered.evaluate_dU(LAY, OMEGA, lam, gamma, dm, zs)[0] / gd
        assert abs(du - dd) < 1e-6 * abs(dd), (m, du, dd)
    jump = (layered.evaluate_dU(LAY, OMEGA, lam, gamma, zs + 1e-9, zs)[0]
            - layered.evaluate_dU(LAY, OMEGA, lam, gamma, zs - 1e-9, zs)[0])
    assert abs(jump + 2.0) < 1e-6


def test_U_ode_residual():
    lam, zs, h = 2e-3, 650.0, 1e-2
    for gamma in ["1", "sigma"]:
        for z in [100.0, 500.0, 1000.0, 2000.0]:
            m = int(np.searchsorted(np.asarray(LAY.interfaces), z, side="right"))
            eta2 = lam ** 2 - 1j * OMEGA * layered.MU0 * LAY.sigma[m]
            u = [layered.evaluate_U(LAY, OMEGA, lam, gamma, z + k * h, zs)[0] for k in (-1, 0, 1)]
            d2 = (u[0] - 2 * u[1] + u[2]) / h ** 2
            assert abs(d2 - eta2 * u[1]) < 1e-4 * abs(eta2 * u[1])


def test_U_whole_space_closed_form():
    hom = Layers((0.0, 400.0), (0.1, 0.1, 0.1))
    for lam in [1e-4, 1e-2, 3.0]:
        eta = np.sqrt(lam ** 2 - 1j * OMEGA * layered.MU0 * 0.1)
        for gamma in ["1", "sigma"]:
            for z, zs in [(50.0, 60.0), (700.0, 20.0), (-30.0, 500.0)]:
                u = layered.evaluate_U(hom, OMEGA, lam, gamma, z, zs)[0]
                ref = np.exp(-eta * abs(z - zs)) / eta
                assert abs(u - ref) <= 1e-12 * abs(ref) + 1e-300


def test_U_large_lambda_no_overflow():
    for lam in [10.0, 1e3, 1e5]:
        for gamma in ["1", "sigma"]:
            u = layered.evaluate_U(LAY, OMEGA, lam, gamma, 1499.0, 1501.0)[0]
            assert np.isfinite(u)
            ref = np.exp(-lam * 2.0) / lam
            assert abs(u) <= 2 * abs(ref) + 1e-300


def _brute(layers, omega, lam, gamma, c1, c2):
    f = lambda zs, z: layered.evaluate_U(layers, omega, lam, gamma, z, zs)[0]
    pts = None
    re = integrate.dblquad(lambda zs, z: f(zs, z).real, c1[0], c1[1], c2[0], c2[1], epsabs=0, epsrel=1e-11)[0]
    im = integrate.dblquad(lambda zs, z: f(zs, z).imag, c1[0], c1[1], c2[0], c2[1], epsabs=0, epsrel=1e-11)[0]
    return re + 1j * im


@pytest.mark.parametrize("lam", [1e-4, 5e-3, 4e-2])
def test_vertical_integrals_brute_force(lam):
    """V1, V2, V4, V5 and V3 against direct quadrature of U over the cell pair."""
    z_edges = np.array([0.0, 100.0, 300.0, 450.0, 800.0, 950.0, 1500.0])
    V = layered.vertical_integrals(LAY, OMEGA, z_edges, np.array([lam]))
    lay = layered.cell_layers(LAY, z_edges)
    iwm = 1j * OMEGA * layered.MU0
    for a, b in [(0, 0), (0, 1), (1, 0), (2, 3), (3, 2), (4, 4), (1, 5), (5, 1), (3, 3)]:
        c1 = (z_edges[a], z_edges[a + 1])
        c2 = (z_edges[b], z_edges[b + 1])
        for gamma, key in (("1", "V1"), ("sigma", "V2")):
            if c1 == c2:
                # split the square along the diagonal for the quadrature
                f = lambda zs, z: layered.evaluate_U(LAY, OMEGA, lam, gamma, z, zs)[0]
                tot = 0
                for part in (lambda z: c1[0], lambda z: z), (lambda z: z, lambda z: c1[1]):
                    re = integrate.dblquad(lambda zs, z: f(zs, z).real, c1[0], c1[1], part[0], part[1], epsrel=1e-11)[0]
                    im = integrate.dblquad(lambda zs, z: f(zs, z).imag, c1[0], c1[1], part[0], part[1], epsrel=1e-11)[0]
                    tot += re + 1j * im
                ref = iwm * tot
            else:
                ref = iwm * _brute(LAY, OMEGA, lam, gamma, c1, c2)
            got = V[key][0, a, b]
            assert abs(got - ref) <= 1e-8 * abs(ref), (a, b, key, got, ref)
        sa = LAY.sigma[lay[a]]
        Us = lambda z, zs: layered.evaluate_U(LAY, OMEGA, lam, "sigma", z, zs, r=lay[a], s=lay[b])[0]
        F = lambda z: integrate.quad(lambda zs: Us(z, zs).real, *c2, epsrel=1e-12, points=[z] if c2[0] < z < c2[1] else None)[0] + \
            1j * integrate.quad(lambda zs: Us(z, zs).imag, *c2, epsrel=1e-12, points=[z] if c2[0] < z < c2[1] else None)[0]
        eps = 0.0
        v4 = (F(c1[1] - eps) - F(c1[0] + eps)) / sa
        assert abs(V["V4"][0, a, b] - v4) <= 1e-6 * abs(v4) + 1e-9 * abs(V["V2"][0, a, b] / iwm / sa), (a, b)
        # V5 via the derivative of F by central differences just inside the cell
        # second-order one-sided differences from inside the field cell
        def dF(hs):
            d2 = (3 * F(c1[1]) - 4 * F(c1[1] - hs) + F(c1[1] - 2 * hs)) / (2 * hs)
            d1 = (-3 * F(c1[0]) + 4 * F(c1[0] + hs) - F(c1[0] + 2 * hs)) / (2 * hs)
            return d2 - d1
        hs = 4e-3 * (c1[1] - c1[0])
        v5 = (4 * dF(hs / 2) - dF(hs)) / 3 / sa      # Richardson step on the O(h^2) differences
        assert abs(V["V5"][0, a, b] - v5) <= 2e-5 * abs(v5) + 1e-6, (a, b, V["V5"][0, a, b], v5)
        Uc = lambda z, zs: layered.evaluate_U(LAY, OMEGA, lam, "sigma", z, zs, r=lay[a], s=lay[b])[0]
        v3 = -(Uc(c1[1], c2[1]) - Uc(c1[1], c2[0]) - Uc(c1[0], c2[1]) + Uc(c1[0], c2[0])) / sa
        assert abs(V["V3w"][0, a, b] - v3) <= 1e-10 * abs(v3) + 1e-300
