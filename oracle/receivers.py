"""Fields at receivers, the MT impedance, its misfit and the misfit gradient.

Test infrastructure (see ``oracle/__init__``).  Paper: eq. (APR_lab) (the field at
a point outside the domain from the solution U), Appendix A eqs. (geh),
(green_tensor), (G1G2g), (Ge2) (the electric and magnetic Green's tensors), and
the same vertical (Appendix B) and lateral (Appendix C) machinery as the
coefficients B_n^m.

Receiver r sits at the lateral centre of grid cell (iy, ix), at depth z_r at or
above the top of the grid.  The paper gives (APR_lab) for points outside the
domain; here every source cell must lie strictly below the receiver plane
(top edge > z_r), which keeps all lambda integrals exponentially convergent.
Cells touching the receiver plane get zero kernels, and the caller must keep
their anomaly empty.

Field of a source box m with uniform current J (J_n = (sigma_a - sigma_b) E_n =
2 s_n gamma_n U_n, reading of (APR_lab)), with D = (x_r - x_m, y_r - y_m):

  E_a = sum_b GE_ab J_b,  H_a = sum_b GH_ab J_b   (a in {x, y}, b in {x, y, z})

  4 pi GE_xx = int K_J P1 lam dlam + int K_xx X dlam / lam,  X = P1 + P3
  4 pi GE_yy = int K_J P1 lam dlam + int K_yy X dlam / lam
  4 pi GE_xy = 4 pi GE_yx = int K_xy X dlam / lam
  4 pi GE_xz = int K_x P4 lam dlam,  4 pi GE_yz = int K_y P4 lam dlam
  4 pi GH_xx = -int K_xy Pg dlam / lam = -4 pi GH_yy
  4 pi GH_yx = int K_J P1z lam dlam + int K_xx Pg dlam / lam
  4 pi GH_xy = -int K_J P1z lam dlam - int K_yy Pg dlam / lam
  4 pi GH_xz = int K_y Ps lam dlam,  4 pi GH_yz = -int K_x Ps lam dlam

with K the lateral integrals of J0 over the source rectangle seen from the point
(the box transform h sinc(k h / 2) in place of the tent of the cell-to-cell
kernels; derivatives act on D), and the vertical functions at the receiver depth
(U = U(z_r, z*), integrated over the source cell z* in [w1, w2]):

  P1  = i w mu0 int U_1,          P3 = -(1/sigma_r) d/dz [U_s(z, w2) - U_s(z, w1)],
  P4  = (1/sigma_r) d/dz int U_s,  P1z = d/dz int U_1,
  Pg  = U_s(z_r, w2) - U_s(z_r, w1) + P1z,   Ps = int U_s,

sigma_r the background conductivity at the receiver.  They follow from (Ge2)
(G_1 + dg/dz = (i w mu0/4 pi) int J0 [k^2 U_1 - d/dz d/dz0 U_s] dlam / lam, as
for B) and from GH = (1/(i w mu0)) curl G with the columns of (green_tensor),
whose curls are, with derivatives in the receiver coordinates,
  J_x: (d2g/dxdy, dG1/dz - d2g/dx2, .),  J_y: (d2g/dy2 - dG1/dz, -d2g/dxdy, .),
  J_z: (dG2/dy, -dG2/dx, .).

The normal field at the receivers is the 1-D field of ``normal``: for the
x-polarisation E_x = E^N(z_r), H_y = E^N'(z_r) / (i w mu0) (= 1 at the surface),
for the y-polarisation E_y = E^N(z_r), H_x = -E^N'(z_r) / (i w mu0).

Impedance (two polarisations per frequency): E = Z H with the 2x2 matrices
E = [[Ex1, Ex2], [Ey1, Ey2]], H = [[Hx1, Hx2], [Hy1, Hy2]], so Z = E H^-1.
Misfit: Phi = 1/2 sum over frequencies, receivers and the four entries of
|Z - Z_obs|^2.

Gradient with respect to theta_m = ln sigma_a^m over the anomalous cells
(gamma_m != 0).  The adjoint of the chain theta -> gamma -> U -> J -> (E, H) -> Z
gives, with D_r = conj(Z_r - Zobs_r), M_r = H_r^-1 D_r^T and for polarisation j
the receiver sources c^E_i = (M_r)_{ji}, c^H_i = -(M_r Z_r)_{ji}:
  q = sum_r GE_r^T c^E_r + GH_r^T c^H_r          (per cell, 3 components)
  A^T w = 2 s gamma q                             (adjoint solve; A^T = S + R2 B R1)
  dPhi/dtheta_m = Re sum_{f, j} (dgamma_m/dtheta_m) (w_m . U_m) / gamma_m
(the terms through J's explicit gamma and through B cancel against the transpose
equation), dgamma/dsigma_a = 2 Re sigma_b / (sigma_a + conj sigma_b)^2 and
dsigma_a/dtheta = sigma_a.  ``gradient_general`` evaluates the uncancelled form
with the dense B for the check.

Pins (tests/test_oracle_receivers.py): the homogeneous whole space against a
brute-force cubature of i w mu0 (I + grad grad / k^2) e^{ikR}/(4 pi R) and of
grad(e^{ikR}/(4 pi R)) x J over the box; continuity of the tangential E and H
across the surface (air-side against earth-side formulas); the point lateral
kernel against direct quadrature; the 1-D impedance of a model without anomaly;
and the gradient against central finite differences.
"""
from __future__ import annotations

import numpy as np

from . import coefficients, layered, normal, operator

MU0 = 4e-7 * np.pi
FOUR_PI = 4.0 * np.pi


def _box_hat(k, h):
    return h * np.sinc(k * h / (2.0 * np.pi))


def point_lateral_kernels(lam, Dx, Dy, hx, hy):
    """K_J, K_xx, K_yy, K_xy, K_x, K_y of a point at lateral offset D from the centre
    of an hx x hy rectangle: K_J = int_rect J0(lam |D - xi|) dxi and its derivatives
    in D, from the 2-D Fourier form of J0 (trapezoidal rule in the angle)."""
    lam = np.asarray(lam, dtype=np.float64)
    out = {k: np.zeros(lam.shape[0]) for k in ("J", "xx", "yy", "xy", "x", "y")}
    for n, L in enumerate(lam):
        nt = int(np.ceil(0.32 * L * (abs(Dx) + abs(Dy) + hx + hy))) + 24
        t = np.linspace(0.0, 0.5 * np.pi, nt + 1)
        w = np.full(nt + 1, 1.0 / nt)
        w[0] *= 0.5
        w[-1] *= 0.5
        kx, ky = L * np.cos(t), L * np.sin(t)
        base = _box_hat(kx, hx) * _box_hat(ky, hy) * w
        cx, sx, cy, sy = np.cos(kx * Dx), np.sin(kx * Dx), np.cos(ky * Dy), np.sin(ky * Dy)
        bcc = base * cx * cy
        out["J"][n] = bcc.sum()
        out["xx"][n] = -(kx * kx * bcc).sum()
        out["yy"][n] = -(ky * ky * bcc).sum()
        out["xy"][n] = (kx * ky * base * sx * sy).sum()
        out["x"][n] = -(kx * base * sx * cy).sum()
        out["y"][n] = -(ky * base * cx * sy).sum()
    return out


def receiver_layer(layers, z_r):
    """Layer index of the receiver depth (the layer below when on an interface)."""
    d = np.asarray(layers.interfaces, dtype=np.float64)
    return int(np.searchsorted(d, z_r, side="right"))


def point_vertical(layers, omega, z_r, z_edges, lam, r=None):
    """P1, X = P1 + P3, P4, P1z, Pg, Ps (dict of arrays [n_lam][Nz]) for the receiver
    depth z_r (in layer r) and every source cell; zero for cells not strictly below
    the receiver."""
    z_edges = np.asarray(z_edges, dtype=np.float64)
    nz = len(z_edges) - 1
    lay = layered.cell_layers(layers, z_edges)
    sig = np.asarray(layers.sigma, dtype=np.complex128)
    r = receiver_layer(layers, z_r) if r is None else r
    lam = np.asarray(lam, dtype=np.float64)
    s1 = layered.Spectrum(layers, omega, lam, "1")
    ss = layered.Spectrum(layers, omega, lam, "sigma")
    out = {k: np.zeros((lam.shape[0], nz), dtype=np.complex128) for k in ("P1", "X", "P4", "P1z", "Pg", "Ps")}
    iwm = 1j * omega * MU0
    inv = 1.0 / sig[r]
    for b in range(nz):
        w1, w2, s = z_edges[b], z_edges[b + 1], lay[b]
        if not w1 > z_r:
            continue
        t1 = s1.terms(r, s, False)
        ts = ss.terms(r, s, False)
        F1 = layered._F(t1, z_r, w1, w2)
        F1z = layered._F(t1, z_r, w1, w2, True)
        Fs = layered._F(ts, z_r, w1, w2)
        Fsz = layered._F(ts, z_r, w1, w2, True)
        dU = 0.0
        Ud = 0.0
        for c, a, bb, k, _ in ts:
            e2 = c * np.exp(a * z_r + bb * w2 + k)
            e1 = c * np.exp(a * z_r + bb * w1 + k)
            dU = dU + a * (e2 - e1)
            Ud = Ud + (e2 - e1)
        P1 = iwm * F1
        P3 = -inv * dU
        out["P1"][:, b] = P1
        out["X"][:, b] = P1 + P3
        out["P4"][:, b] = inv * Fsz
        out["P1z"][:, b] = F1z
        out["Pg"][:, b] = Ud + F1z
        out["Ps"][:, b] = Fs
    return out


def receiver_kernels_offset(grid, layers, freq, z_r, Dx, Dy, r=None):
    """GE, GH (each [Nz][2][3]: receiver component x/y, source component x/y/z) for a
    receiver at lateral offset D from the source cells' centres."""
    z_edges = grid.z_edges_array()
    hx, hy = grid.hx, grid.hy
    hmin = min(hx, hy, float(np.min(np.diff(z_edges))))
    omega = 2.0 * np.pi * freq
    lam, w, _ = coefficients.lambda_nodes(Dx, Dy, hx, hy, hmin)
    K = point_lateral_kernels(lam, Dx, Dy, hx, hy)
    P = point_vertical(layers, omega, z_r, z_edges, lam, r)
    wl = (w * lam)[:, None]
    wi = (w / lam)[:, None]
    kJ, kxx, kyy, kxy, kx, ky = (K[n][:, None] for n in ("J", "xx", "yy", "xy", "x", "y"))

    def I(wt, k, f):
        return np.sum(wt * k * P[f], 0)
    nz = grid.nz
    GE = np.zeros((nz, 2, 3), dtype=np.complex128)
    GH = np.zeros((nz, 2, 3), dtype=np.complex128)
    JP1 = I(wl, kJ, "P1")
    GE[:, 0, 0] = JP1 + I(wi, kxx, "X")
    GE[:, 1, 1] = JP1 + I(wi, kyy, "X")
    GE[:, 0, 1] = GE[:, 1, 0] = I(wi, kxy, "X")
    GE[:, 0, 2] = I(wl, kx, "P4")
    GE[:, 1, 2] = I(wl, ky, "P4")
    hxy = I(wi, kxy, "Pg")
    JP1z = I(wl, kJ, "P1z")
    GH[:, 0, 0] = -hxy
    GH[:, 1, 1] = hxy
    GH[:, 1, 0] = JP1z + I(wi, kxx, "Pg")
    GH[:, 0, 1] = -JP1z - I(wi, kyy, "Pg")
    GH[:, 0, 2] = I(wl, ky, "Ps")
    GH[:, 1, 2] = -I(wl, kx, "Ps")
    return GE / FOUR_PI, GH / FOUR_PI


def receiver_operator(grid, layers, freq, z_r, receivers):
    """Dense receiver operator G [n_rec][4][3 N]: rows (Ex, Ey, Hx, Hy) of each
    receiver, columns the current J in the layout [3][Nz][Ny][Nx]; every
    (receiver, cell) offset computed directly."""
    nx, ny, nz = grid.nx, grid.ny, grid.nz
    N = nx * ny * nz
    G = np.zeros((len(receivers), 4, 3 * N), dtype=np.complex128)
    cache = {}
    for ir, (iy, ix) in enumerate(receivers):
        for i in range(ny):
            for j in range(nx):
                key = (iy - i, ix - j)
                if key not in cache:
                    cache[key] = receiver_kernels_offset(grid, layers, freq, z_r, key[1] * grid.hx, key[0] * grid.hy)
                GE, GH = cache[key]
                for b in range(nz):
                    cell = (b * ny + i) * nx + j
                    for c in range(3):
                        G[ir, 0:2, c * N + cell] = GE[b, :, c]
                        G[ir, 2:4, c * N + cell] = GH[b, :, c]
    return G


def receiver_operator_sites(grid, layers, freq, z_r, sites):
    """Dense receiver operator G [n_rec][4][3 N] for receivers at arbitrary lateral
    sites (x, y) in metres, the grid's frame (cell j spans [j hx, (j + 1) hx]): every
    (site, cell) offset from the site to the cell centre computed directly (field
    recovery at any point, eq. (APR_lab))."""
    nx, ny, nz = grid.nx, grid.ny, grid.nz
    N = nx * ny * nz
    G = np.zeros((len(sites), 4, 3 * N), dtype=np.complex128)
    cache = {}
    for ir, (x, y) in enumerate(sites):
        for i in range(ny):
            for j in range(nx):
                Dx, Dy = x - (j + 0.5) * grid.hx, y - (i + 0.5) * grid.hy
                key = (round(Dx, 9), round(Dy, 9))
                if key not in cache:
                    cache[key] = receiver_kernels_offset(grid, layers, freq, z_r, Dx, Dy)
                GE, GH = cache[key]
                for b in range(nz):
                    cell = (b * ny + i) * nx + j
                    for c in range(3):
                        G[ir, 0:2, c * N + cell] = GE[b, :, c]
                        G[ir, 2:4, c * N + cell] = GH[b, :, c]
    return G


def apparent(Z, freq):
    """The MT maps of impedances Z [...][2][2]: apparent resistivity |Z|^2 / (w mu0) in
    ohm m and phase arg Z in degrees."""
    omega = 2.0 * np.pi * freq
    return np.abs(Z) ** 2 / (omega * MU0), np.degrees(np.angle(Z))


def normal_at(layers, freq, z_r):
    """(E^N(z_r), E^N'(z_r) / (i w mu0)) of the 1-D profile."""
    omega = 2.0 * np.pi * freq
    d, kap, coef, row = normal._profile_coefs(layers, omega)
    L = len(d)
    m = min(max(int(np.searchsorted(d, z_r, side="right")), 1), L)
    E = row(m, z_r, False) @ coef
    dE = row(m, z_r, True) @ coef
    return E, dE / (1j * omega * MU0)


def fields(model, freq, U, G, z_r):
    """F [2][n_rec][4] = (Ex, Ey, Hx, Hy) for the x- and y-polarisation solutions
    U [2][3][Nz][Ny][Nx]: normal field plus G J with J = 2 s gamma U."""
    gamma, s, V = operator.diagonals(model)
    En, Hn = normal_at(model.layers, freq, z_r)
    out = np.empty((2, G.shape[0], 4), dtype=np.complex128)
    for p in range(2):
        J = (2.0 * s[:, None, None] * gamma)[None] * U[p]
        out[p] = G @ J.ravel()
    out[0, :, 0] += En
    out[0, :, 3] += Hn
    out[1, :, 1] += En
    out[1, :, 2] -= Hn
    return out


def impedance(F):
    """Z [n_rec][2][2] = E H^-1 from the two polarisations' fields F [2][n_rec][4]."""
    E = np.stack([F[:, :, 0], F[:, :, 1]], axis=1).transpose(2, 1, 0)   # [rec][comp][pol]
    H = np.stack([F[:, :, 2], F[:, :, 3]], axis=1).transpose(2, 1, 0)
    return E @ np.linalg.inv(H)


def misfit(Z, Zobs):
    return 0.5 * float(np.sum(np.abs(Z - Zobs) ** 2))


def with_sigma(model, sigma_a):
    from workloads import Model
    return Model(model.name, model.grid, model.layers, sigma_a, model.freqs, model.pols)


def dense_A(model, qa):
    return operator.dense_matrix(model, operator.dense_B(model, qa))


def solve_pols(model, freq, A):
    from . import normal as nm
    b = np.stack([nm.rhs_U0(model, freq, "x"), nm.rhs_U0(model, freq, "y")])
    return np.stack([np.linalg.solve(A, b[p].ravel()).reshape(b[p].shape) for p in range(2)])


def misfit_of(model, problems, Zobs):
    """Phi summed over frequencies; problems: list of (freq, qa, G, z_r)."""
    phi = 0.0
    for (freq, qa, G, z_r), zo in zip(problems, Zobs):
        U = solve_pols(model, freq, dense_A(model, qa))
        phi += misfit(impedance(fields(model, freq, U, G, z_r)), zo)
    return phi


def adjoint_sources(F, Z, Zobs):
    """c [2][n_rec][4] (receiver-side adjoint sources per polarisation)."""
    E = np.stack([F[:, :, 0], F[:, :, 1]], axis=1).transpose(2, 1, 0)
    H = np.stack([F[:, :, 2], F[:, :, 3]], axis=1).transpose(2, 1, 0)
    D = np.conj(Z - Zobs)
    M = np.linalg.inv(H) @ D.transpose(0, 2, 1)        # H^-1 D^T
    MZ = M @ Z
    c = np.zeros((2, F.shape[1], 4), dtype=np.complex128)
    for j in range(2):
        c[j, :, 0] = M[:, j, 0]
        c[j, :, 1] = M[:, j, 1]
        c[j, :, 2] = -MZ[:, j, 0]
        c[j, :, 3] = -MZ[:, j, 1]
    return c


def gradient(model, problems, Zobs):
    """dPhi/dtheta [Nz][Ny][Nx] (theta = ln sigma_a), zero where gamma = 0."""
    gamma, s, V = operator.diagonals(model)
    from workloads import background_sigma
    sig_b = background_sigma(model.grid, model.layers)[:, None, None] * np.ones_like(model.sigma_a)
    sa = model.sigma_a
    dg = sa * 2.0 * sig_b.real / (sa + np.conj(sig_b)) ** 2
    grad = np.zeros(sa.shape)
    an = gamma != 0
    for (freq, qa, G, z_r), zo in zip(problems, Zobs):
        A = dense_A(model, qa)
        U = solve_pols(model, freq, A)
        F = fields(model, freq, U, G, z_r)
        Z = impedance(F)
        c = adjoint_sources(F, Z, zo)
        for p in range(2):
            q = (G.reshape(-1, G.shape[-1]).T @ c[p].ravel()).reshape(U[p].shape)
            rhs = (2.0 * s[:, None, None] * gamma)[None] * q
            w = np.linalg.solve(A.T, rhs.ravel()).reshape(q.shape)
            wu = np.sum(w * U[p], 0)
            g = np.zeros(sa.shape, dtype=np.complex128)
            g[an] = dg[an] * wu[an] / gamma[an]
            grad += g.real
    return grad


def gradient_general(model, problems, Zobs):
    """The same gradient from the uncancelled adjoint form (every term kept, dense B):
    dPhi/dtheta_m = Re sum dgamma_m [2 s_m q_m.U_m + w_m.U_m - s_m (B R1 w)_m.U_m]."""
    gamma, s, V = operator.diagonals(model)
    from workloads import background_sigma
    sig_b = background_sigma(model.grid, model.layers)[:, None, None] * np.ones_like(model.sigma_a)
    sa = model.sigma_a
    dg = sa * 2.0 * sig_b.real / (sa + np.conj(sig_b)) ** 2
    N = sa.size
    sv = np.tile(np.broadcast_to(s[:, None, None], sa.shape).ravel(), 3)
    R1 = np.tile(np.broadcast_to((-2.0 * s / V)[:, None, None], sa.shape).ravel(), 3)
    grad = np.zeros(sa.shape)
    for (freq, qa, G, z_r), zo in zip(problems, Zobs):
        B = operator.dense_B(model, qa)
        A = operator.dense_matrix(model, B)
        U = solve_pols(model, freq, A)
        F = fields(model, freq, U, G, z_r)
        Z = impedance(F)
        c = adjoint_sources(F, Z, zo)
        for p in range(2):
            qv = G.reshape(-1, G.shape[-1]).T @ c[p].ravel()
            gv = np.tile(gamma.ravel(), 3)
            w = np.linalg.solve(A.T, 2.0 * sv * gv * qv)
            BR1w = B @ (R1 * w)
            uv = U[p].ravel()
            t = (2.0 * sv * qv * uv + w * uv - sv * BR1w * uv).reshape(3, N).sum(0).reshape(sa.shape)
            grad += (dg * t).real
    return grad
