"""Magnetotelluric normal field E^N and the right-hand side U^0.

Test infrastructure (see ``oracle/__init__``).  The paper uses plane-wave (MT)
sources (Sect. 4) but prints no formula for E^N; the plain definition used here
is the 1-D solution of eq. (Maxwell2) in the layered background: with e^{-i w t}
and z downwards, E'' = -i w mu0 sigma_b(z) E, E and E' continuous across the
interfaces, E decaying in the basement, normalised by H(0) = 1 for the source
polarisation (x-polarisation: E = (E, 0, 0), H_y(0) = 1, i.e. E'(0) = i w mu0;
y-polarisation: E = (0, E, 0), H_x(0) = -1, which gives the same profile).

U^0_n = (sqrt(Re sigma_b^n) / V_n) int_{Omega_n} E^N   (eq. (slae_matricies)).

Pins: homogeneous half-space (apparent resistivity 1/sigma, |phase| = 45 deg),
the ODE and continuity conditions (tests/test_oracle_operator.py).
"""
from __future__ import annotations

import numpy as np

MU0 = 4e-7 * np.pi


def _profile_coefs(layers, omega):
    d = np.asarray(layers.interfaces, dtype=np.float64)
    sig = np.asarray(layers.sigma, dtype=np.complex128)
    L = len(d)
    kap = np.sqrt(-1j * omega * MU0 * sig)            # Re > 0
    # unknowns: (a_m, b_m) for finite layers m = 1..L-1, a_L for the basement
    n = 2 * (L - 1) + 1
    A = np.zeros((n, n), dtype=np.complex128)
    rhs = np.zeros(n, dtype=np.complex128)

    def ia(m):
        return 2 * (m - 1)

    def ib(m):
        return 2 * (m - 1) + 1

    def row(m, z, deriv):
        r = np.zeros(n, dtype=np.complex128)
        k = kap[m]
        if m == L:
            v = np.exp(-k * (z - d[L - 1]))
            r[ia(m)] = -k * v if deriv else v
        else:
            top, bot = d[m - 1], d[m]
            va = np.exp(-k * (z - top))
            vb = np.exp(-k * (bot - z))
            r[ia(m)] = -k * va if deriv else va
            r[ib(m)] = k * vb if deriv else vb
        return r
    eq = 0
    A[eq] = row(1, d[0], True)
    rhs[eq] = 1j * omega * MU0
    eq += 1
    for m in range(1, L):
        z = d[m]
        A[eq] = row(m, z, False) - row(m + 1, z, False)
        eq += 1
        A[eq] = row(m, z, True) - row(m + 1, z, True)
        eq += 1
    coef = np.linalg.solve(A, rhs)
    return d, kap, coef, row


def field(layers, omega, z):
    """E^N(z) for z >= 0 (x-polarisation profile)."""
    d, kap, coef, row = _profile_coefs(layers, omega)
    L = len(d)
    out = []
    for zz in np.atleast_1d(z):
        m = min(max(int(np.searchsorted(d, zz, side="right")), 1), L)
        out.append(row(m, zz, False) @ coef)
    return np.array(out)


def cell_average(layers, omega, z1, z2):
    """(1/(z2-z1)) int_{z1}^{z2} E^N dz for a cell inside one layer."""
    d, kap, coef, row = _profile_coefs(layers, omega)
    L = len(d)
    m = min(max(int(np.searchsorted(d, 0.5 * (z1 + z2), side="right")), 1), L)
    k = kap[m]
    h = z2 - z1
    # int e^{-k(z-top)} dz = (e^{-k(z1-top)} - e^{-k(z2-top)}) / k, etc.
    if m == L:
        top = d[L - 1]
        val = coef[2 * (m - 1)] * (np.exp(-k * (z1 - top)) - np.exp(-k * (z2 - top))) / k
    else:
        top, bot = d[m - 1], d[m]
        val = (coef[2 * (m - 1)] * (np.exp(-k * (z1 - top)) - np.exp(-k * (z2 - top))) / k
               + coef[2 * (m - 1) + 1] * (np.exp(-k * (bot - z2)) - np.exp(-k * (bot - z1))) / k)
    return val / h


def surface_impedance(layers, omega):
    """E^N(0) / H(0): the 1-D MT impedance of the background."""
    return field(layers, omega, [0.0])[0]


def rhs_U0(model, freq, pol):
    """U^0 as an array [3][Nz][Ny][Nx] for polarisation 'x' or 'y'."""
    g = model.grid
    ze = g.z_edges_array()
    omega = 2 * np.pi * freq
    from workloads import background_sigma
    sb = background_sigma(g, model.layers)
    avg = np.array([cell_average(model.layers, omega, ze[k], ze[k + 1]) for k in range(g.nz)])
    s = np.sqrt(sb.real)
    out = np.zeros((3, g.nz, g.ny, g.nx), dtype=np.complex128)
    c = 0 if pol == "x" else 1
    out[c] = (s * avg)[:, None, None]
    return out
