"""Pins of the oracle's receiver fields, MT impedance and misfit gradient
(oracle/receivers.py) against things it does not compute itself."""
import numpy as np
import pytest
from scipy import special

import workloads as W
from oracle import coefficients, normal, receivers as RC

MU0 = 4e-7 * np.pi


def _gl(n, a, b):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (b - a) * x + 0.5 * (a + b), 0.5 * (b - a) * w


@pytest.mark.parametrize("lam,Dx,Dy", [(0.003, 0.0, 0.0), (0.02, 150.0, -50.0), (0.05, -100.0, 200.0)])
def test_point_lateral_kernel_direct_quadrature(lam, Dx, Dy):
    """K_J = int over the source rectangle of J0(lam |D - xi|), by 2-D Gauss-Legendre
    quadrature (the rectangle does not contain D away from zero offset; at zero
    offset J0 is smooth anyway), and K_x, K_xx by finite differences in Dx."""
    hx, hy = 100.0, 80.0
    xs, wx = _gl(40, -hx / 2, hx / 2)
    ys, wy = _gl(40, -hy / 2, hy / 2)

    def direct(dx, dy):
        X, Y = np.meshgrid(xs, ys, indexing="ij")
        return float(np.sum(wx[:, None] * wy[None, :] * special.j0(lam * np.hypot(dx - X, dy - Y))))
    K = RC.point_lateral_kernels([lam], Dx, Dy, hx, hy)
    assert abs(K["J"][0] - direct(Dx, Dy)) <= 1e-9 * hx * hy
    e = 1e-2
    kx_fd = (direct(Dx + e, Dy) - direct(Dx - e, Dy)) / (2 * e)
    kxx_fd = (direct(Dx + e, Dy) - 2 * direct(Dx, Dy) + direct(Dx - e, Dy)) / e ** 2
    ky_fd = (direct(Dx, Dy + e) - direct(Dx, Dy - e)) / (2 * e)
    assert abs(K["x"][0] - kx_fd) <= 1e-6 * lam * hx * hy + 1e-9
    assert abs(K["y"][0] - ky_fd) <= 1e-6 * lam * hx * hy + 1e-9
    assert abs(K["xx"][0] - kxx_fd) <= 1e-4 * lam * lam * hx * hy + 1e-9


def _whole_space_reference(omega, sig, Dx, Dy, z_r, hx, hy, w1, w2, n=24):
    """GE, GH [2][3] of a uniform-current box in a homogeneous medium by cubature of
    i w mu0 (I + grad grad / k^2) g0 and grad g0 x J, g0 = e^{ikR}/(4 pi R)."""
    k = np.sqrt(1j * omega * MU0 * sig)
    if k.imag < 0:
        k = -k
    xs, wx = _gl(n, -hx / 2, hx / 2)
    ys, wy = _gl(n, -hy / 2, hy / 2)
    zs, wz = _gl(n, w1, w2)
    X, Y, Z = np.meshgrid(xs, ys, zs, indexing="ij")
    Wt = wx[:, None, None] * wy[None, :, None] * wz[None, None, :]
    Rv = np.stack([Dx - X, Dy - Y, z_r - Z])          # receiver minus source point
    R = np.sqrt(np.sum(Rv ** 2, 0))
    u = Rv / R
    g0 = np.exp(1j * k * R) / (4 * np.pi * R)
    g1 = (1j * k - 1.0 / R) * g0                      # d g0 / dR
    g2 = ((1j * k - 1.0 / R) ** 2 + 1.0 / R ** 2) * g0
    GE = np.zeros((2, 3), dtype=np.complex128)
    GH = np.zeros((2, 3), dtype=np.complex128)
    grad = u * g1
    for a in range(2):
        for b in range(3):
            dd = u[a] * u[b] * g2 + ((1.0 if a == b else 0.0) - u[a] * u[b]) * g1 / R
            val = (g0 if a == b else 0.0) + dd / k ** 2
            GE[a, b] = 1j * omega * MU0 * np.sum(Wt * val)
    eps = np.zeros((3, 3, 3))
    eps[0, 1, 2] = eps[1, 2, 0] = eps[2, 0, 1] = 1.0
    eps[0, 2, 1] = eps[2, 1, 0] = eps[1, 0, 2] = -1.0
    for a in range(2):
        for b in range(3):
            GH[a, b] = sum(eps[a, c, b] * np.sum(Wt * grad[c]) for c in range(3))
    return GE, GH


@pytest.mark.parametrize("D", [(0.0, 0.0), (100.0, 0.0), (100.0, -200.0)])
def test_whole_space_receiver_kernels(D):
    """Homogeneous medium (air and earth at one conductivity): the receiver kernels
    equal the cubature of the textbook dyadic Green's function and its curl."""
    sig = 0.05
    layers = W.Layers((0.0,), (sig, sig))
    grid = W.uniform_grid(2, 2, 2, 100.0, z0=100.0)
    freq = 3.0
    GE, GH = RC.receiver_kernels_offset(grid, layers, freq, 0.0, D[0], D[1])
    ze = grid.z_edges_array()
    for b in range(grid.nz):
        ge, gh = _whole_space_reference(2 * np.pi * freq, sig, D[0], D[1], 0.0, 100.0, 100.0, ze[b], ze[b + 1])
        scale_e = np.max(np.abs(ge))
        scale_h = np.max(np.abs(gh))
        assert np.max(np.abs(GE[b] - ge)) <= 1e-6 * scale_e, (b, GE[b], ge)
        assert np.max(np.abs(GH[b] - gh)) <= 1e-6 * scale_h, (b, GH[b], gh)


def test_tangential_fields_continuous_across_the_surface():
    """E_x, E_y, H_x, H_y at z = 0 from the air-side formulas (receiver layer 0) equal
    those from the earth side (layer 1): the kernels carry the interface
    conditions of U_1 and U_sigma, including the 1/sigma_r factors."""
    layers = W.Layers((0.0, 150.0, 400.0), (1e-6, 0.02, 0.2, 0.005))
    grid = W.uniform_grid(2, 2, 3, 100.0, z0=50.0)
    for D in ((0.0, 0.0), (100.0, 100.0)):
        GE0, GH0 = RC.receiver_kernels_offset(grid, layers, 1.0, 0.0, D[0], D[1], r=0)
        GE1, GH1 = RC.receiver_kernels_offset(grid, layers, 1.0, 0.0, D[0], D[1], r=1)
        assert np.max(np.abs(GE0 - GE1)) <= 1e-8 * np.max(np.abs(GE1))
        assert np.max(np.abs(GH0 - GH1)) <= 1e-8 * np.max(np.abs(GH1))


def test_impedance_without_anomaly_is_the_1d_impedance():
    """sigma_a = sigma_b: no current, so Z = [[0, Z1], [-Z1, 0]] with Z1 the 1-D
    surface impedance; for a half-space rho_a = |Z1|^2 / (w mu0) = 1/sigma and the
    phase is 45 degrees."""
    sig = 0.01
    layers = W.Layers((0.0,), (1e-9, sig))
    grid = W.uniform_grid(2, 2, 2, 100.0, z0=100.0)
    sb = W.background_sigma(grid, layers)
    m = W.Model("hs", grid, layers, np.broadcast_to(sb[:, None, None], (2, 2, 2)).astype(np.complex128).copy(),
                (1.0,), ("x", "y"))
    rec = [(0, 0), (1, 1)]
    G = RC.receiver_operator(grid, layers, 1.0, 0.0, rec)
    U = np.stack([normal.rhs_U0(m, 1.0, "x"), normal.rhs_U0(m, 1.0, "y")])
    Z = RC.impedance(RC.fields(m, 1.0, U, G, 0.0))
    Z1 = normal.surface_impedance(layers, 2 * np.pi)
    for z in Z:
        assert abs(z[0, 0]) < 1e-12 and abs(z[1, 1]) < 1e-12
        assert abs(z[0, 1] - Z1) <= 1e-12 * abs(Z1)
        assert abs(z[1, 0] + Z1) <= 1e-12 * abs(Z1)
    omega = 2 * np.pi
    assert abs(abs(Z1) ** 2 / (omega * MU0) * sig - 1.0) < 1e-9
    assert abs(abs(np.angle(Z1, deg=True)) - 45.0) < 1e-7


def _tiny_problem():
    layers = W.Layers((0.0, 150.0), (1e-9, 0.02, 0.005))
    grid = W.uniform_grid(3, 3, 2, 50.0, z0=50.0)
    sb = W.background_sigma(grid, layers)
    sa = np.broadcast_to(sb[:, None, None], (2, 3, 3)).astype(np.complex128).copy()
    sa[0, 1, 1] = 0.5
    sa[1, 1, 2] = 0.3
    sa[1, 0, 0] = 0.001
    m = W.Model("rx_tiny", grid, layers, sa, (1.0, 10.0), ("x", "y"))
    rec = [(0, 0), (1, 1), (2, 1), (0, 2)]
    problems = []
    for f in m.freqs:
        qa = coefficients.all_offsets(grid, layers, f)
        G = RC.receiver_operator(grid, layers, f, 0.0, rec)
        problems.append((f, qa, G, 0.0))
    rng = np.random.default_rng(5)
    zobs = []
    for (f, qa, G, zr) in problems:
        U = RC.solve_pols(m, f, RC.dense_A(m, qa))
        Z = RC.impedance(RC.fields(m, f, U, G, zr))
        zobs.append(Z * (1.0 + 0.05 * (rng.standard_normal(Z.shape) + 1j * rng.standard_normal(Z.shape))))
    return m, problems, zobs


def test_gradient_against_finite_differences():
    """The cancelled adjoint gradient equals the uncancelled form (dense B) and
    central finite differences in ln sigma_a (h = 1e-4) on every anomalous cell."""
    m, problems, zobs = _tiny_problem()
    g = RC.gradient(m, problems, zobs)
    g2 = RC.gradient_general(m, problems, zobs)
    an = np.argwhere(np.abs(m.sigma_a - W.background_sigma(m.grid, m.layers)[:, None, None]) > 0)
    assert len(an) == 3
    for idx in map(tuple, an):
        assert abs(g[idx] - g2[idx]) <= 1e-9 * max(abs(g2[idx]), 1e-30), (idx, g[idx], g2[idx])
        h = 1e-4
        sp = m.sigma_a.copy(); sp[idx] *= np.exp(h)
        sm = m.sigma_a.copy(); sm[idx] *= np.exp(-h)
        fd = (RC.misfit_of(RC.with_sigma(m, sp), problems, zobs) - RC.misfit_of(RC.with_sigma(m, sm), problems, zobs)) / (2 * h)
        assert abs(g[idx] - fd) <= 1e-6 * abs(fd) + 1e-14, (idx, g[idx], fd)
    # away from the anomaly the cancelled form is not defined and is reported as zero
    assert g[0, 2, 2] == 0.0
