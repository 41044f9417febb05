"""Galerkin coefficients B_n^m and the compressed tensor Q(i, j).

Test infrastructure (see ``oracle/__init__``).  Paper: Appendix A (the 3x3 form
of B_n^m in terms of I_1, I_2, I_xx, I_xy, I_yy, I_x, I_y, I_zz, eq. (Hor_Int),
(Ver_Int)), Sect. 3.1 (block-Toeplitz structure (bcyl), (Q_def), the symmetries
(tensor_symm), (tensor_symm_2), (matrix_symm) and the compressed storage).

For field cell n and source cell m with lateral offset D = (j hx, i hy)
(i = I_y^n - I_y^m, j = I_x^n - I_x^m) and z-cells a (of n), b (of m):

  4 pi B_xx = I1 + Ixx,  4 pi B_yy = I1 + Iyy,  4 pi B_zz = I2 + Izz,
  4 pi B_xy = Ixy,       4 pi B_xz = Ix,        4 pi B_yz = Iy,
  B_zx(D)[a, b] = -B_xz(D)[b, a],  B_zy(D)[a, b] = -B_yz(D)[b, a]   (Lemma 1),

  I1  = int K_J  V1 lam dlam,             I2  = int K_J  V2 lam dlam,
  Izz = int K_J  V5 lam dlam,             Ix  = int K_x  V4 lam dlam,
  Ixx = int K_xx (V1 + V3) dlam / lam     (and yy, xy likewise),

with the lateral kernels K of ``lateral`` and the vertical integrals V of
``layered``.

Readings of the paper used here:
* V3 in Ixx, Iyy, Ixy is the classical derivative: the delta of
  d/dz d/dz* U_sigma at z = z* is excluded, i.e. V3 = V3w + (2/sigma_a) |a cap b|
  with V3w the cell-face (nested-integral) value.  Only then does
  (V1 + V3)/lambda^2 equal (1/sigma) int int U in the homogeneous whole space,
  as G_1 + dg/dz requires; the whole-space test pins it.
* The zx, zy blocks follow Lemma 1; the reciprocity remark under eq. (Ge2)
  (G_xz(M,M0) = -G_zx(M0,M)) would give the opposite sign; the whole-space
  test pins Lemma 1's sign.
* Lambda quadrature (Appendix C computes the same integrals with a digital
  filter whose output functions are not printed): for cells whose lateral
  footprints touch or overlap (|i|, |j| <= 1) the quasi-static part of the
  U_sigma kinds (V3, V4, V5), whose lambda integrals converge only
  algebraically, is subtracted and added back in closed form (``static``);
  the remainder is integrated with Gauss-Legendre panels up to lambda h = 300.
  For separated footprints the integrand oscillates with frequency at least
  the footprint gap R_min and is integrated under a smooth window
  0.5 erfc((lam - 80/R_min) / (10/R_min)), whose error is of order
  exp(-25).

Parity: pinned (homogeneous whole-space brute force; lateral, vertical and
static parts pinned separately; symmetries and the contraction bound).
"""
from __future__ import annotations

import numpy as np
from scipy import special

from . import lateral, layered, static

FOUR_PI = 4.0 * np.pi
NEAR_LH = 300.0          # lambda * h_min reached for touching footprints
FAR_C, FAR_W = 80.0, 10.0
GL_N = 8
PANEL_REL = 0.25
LAM_LOW = 1e-9


def _gl_panels(edges, n=GL_N):
    x, w = np.polynomial.legendre.leggauss(n)
    a, b = edges[:-1, None], edges[1:, None]
    return (0.5 * (b - a) * x[None, :] + 0.5 * (a + b)).ravel(), (0.5 * (b - a) * w[None, :]).ravel()


def lambda_nodes(Dx, Dy, hx, hy, hmin):
    """Quadrature nodes, weights (window included) and the near flag for one offset.

    Gauss-Legendre panels whose width is min(PANEL_REL * lam, pi / rmax): relative
    (logarithmic) panels resolve the branch points of eta_m = sqrt(lam^2 - k_m^2)
    at lam = k_m, whose distance from the real axis is of the order of lam there;
    the absolute cap resolves the oscillation of the lateral kernels, whose
    frequency is at most rmax."""
    rmax = np.hypot(abs(Dx) + hx, abs(Dy) + hy)
    near = abs(Dx) <= hx * (1 + 1e-12) and abs(Dy) <= hy * (1 + 1e-12)
    if near:
        lam_end = NEAR_LH / hmin
        rmin = 0.0
    else:
        rmin = np.hypot(max(abs(Dx) - hx, 0.0), max(abs(Dy) - hy, 0.0))
        lam_end = (FAR_C + 6.0 * FAR_W) / rmin
    edges = [LAM_LOW]
    cap = np.pi / rmax
    while edges[-1] < lam_end:
        edges.append(min(lam_end, edges[-1] + min(PANEL_REL * edges[-1], cap)))
    lam, w = _gl_panels(np.asarray(edges))
    if not near:
        w = w * 0.5 * special.erfc((lam - FAR_C / rmin) / (FAR_W / rmin))
    return lam, w, near


def _static_blocks(Dx, Dy, hx, hy, z_edges, lay, sig, d_ext):
    """Closed-form static parts S_kind[a, b] (kinds xx, yy, xy, xz, yz, zz).

    The static U_sigma is c e^{-lam|z-z*|}/lam plus, within one layer, the images
    P_top e^{-lam(z+z*-2 d_r)}/lam and P_bot e^{-lam(2 d_{r+1}-z-z*)}/lam.  In space an
    image is 1/r to the source box mirrored in the interface.  Under -d/dz d/dz*
    (the V3 kinds xx, yy, xy) an image changes sign; under d/dz and d2/dz2 (V4, V5:
    xz, yz, zz) it does not."""
    nz = len(z_edges) - 1
    spec = layered.StaticSpectrum.__new__(layered.StaticSpectrum)
    spec.sig, spec.L = sig, len(sig) - 1
    out = {k: np.zeros((nz, nz), dtype=np.complex128) for k in ("xx", "yy", "xy", "xz", "yz", "zz")}
    for a in range(nz):
        z1, z2, r = z_edges[a], z_edges[a + 1], lay[a]
        for b in range(nz):
            w1, w2, s = z_edges[b], z_edges[b + 1], lay[b]
            c, pt, pb = layered.StaticSpectrum.coefs(spec, r, s)
            if c == 0.0:
                continue
            boxes = [(c, False, w1, w2)]
            if r == s and pt != 0.0:
                boxes.append((pt, True, 2 * d_ext[r] - w2, 2 * d_ext[r] - w1))
            if r == s and pb != 0.0:
                boxes.append((pb, True, 2 * d_ext[r + 1] - w2, 2 * d_ext[r + 1] - w1))
            for kind in out:
                acc = 0.0
                for coef, image, s1, s2 in boxes:
                    sgn = -1.0 if (image and kind in ("xx", "yy", "xy")) else 1.0
                    acc = acc + sgn * coef * static.box_d2(kind, Dx, Dy, hx, hy, z1, z2, s1, s2)
                out[kind][a, b] = acc / sig[r]
    return out


def offset_blocks(grid, layers, freq, i, j):
    """The six independent Nz x Nz blocks (xx, yy, zz, xy, xz, yz) of Q(i, j)."""
    z_edges = grid.z_edges_array()
    hx, hy = grid.hx, grid.hy
    Dx, Dy = j * hx, i * hy
    hmin = min(hx, hy, float(np.min(np.diff(z_edges))))
    omega = 2.0 * np.pi * freq
    lam, w, near = lambda_nodes(Dx, Dy, hx, hy, hmin)
    K = lateral.lateral_kernels(lam, Dx, Dy, hx, hy)
    V = layered.vertical_integrals(layers, omega, z_edges, lam)
    lay = layered.cell_layers(layers, z_edges)
    sig = np.asarray(layers.sigma, dtype=np.complex128)
    nz = grid.nz
    ovl = np.diag(np.diff(z_edges))                          # |a cap b|
    inv_sig = 1.0 / sig[lay]                                 # per field cell a
    V3p = V["V3w"] + (2.0 * inv_sig[:, None] * ovl)[None]
    V3 = V3p
    V4, V5 = V["V4"], V["V5"]
    if near:
        Vs = layered.vertical_integrals(layers, omega, z_edges, lam, static=True)
        V3 = V["V3w"] - Vs["V3w"]
        V4 = V4 - Vs["V4"]
        V5 = V5 - Vs["V5"]
    wl = (w * lam)[:, None, None]
    wi = (w / lam)[:, None, None]
    kJ, kxx, kyy, kxy, kx, ky = (K[n][:, None, None] for n in ("J", "xx", "yy", "xy", "x", "y"))
    I1 = np.sum(wl * kJ * V["V1"], 0)
    I2 = np.sum(wl * kJ * V["V2"], 0)
    Izz = np.sum(wl * kJ * V5, 0)
    Ix = np.sum(wl * kx * V4, 0)
    Iy = np.sum(wl * ky * V4, 0)
    X = V["V1"] + V3
    Ixx = np.sum(wi * kxx * X, 0)
    Iyy = np.sum(wi * kyy * X, 0)
    Ixy = np.sum(wi * kxy * X, 0)
    if near:
        d = np.asarray(layers.interfaces, dtype=np.float64)
        d_ext = np.concatenate([[d[0]], d, [d[-1]]])
        S = _static_blocks(Dx, Dy, hx, hy, z_edges, lay, sig, d_ext)
        Ixx, Iyy, Ixy = Ixx + S["xx"], Iyy + S["yy"], Ixy + S["xy"]
        Ix, Iy, Izz = Ix + S["xz"], Iy + S["yz"], Izz + S["zz"]
    out = np.empty((6, nz, nz), dtype=np.complex128)
    out[0] = (I1 + Ixx) / FOUR_PI
    out[1] = (I1 + Iyy) / FOUR_PI
    out[2] = (I2 + Izz) / FOUR_PI
    out[3] = Ixy / FOUR_PI
    out[4] = Ix / FOUR_PI
    out[5] = Iy / FOUR_PI
    return out


def full_block(q6):
    """3Nz x 3Nz block [[xx, xy, xz], [xy, yy, yz], [zx, zy, zz]] from the six blocks
    (zx = -xz^T, zy = -yz^T by Lemma 1, yx = xy)."""
    xx, yy, zz, xy, xz, yz = q6
    return np.block([[xx, xy, xz], [xy, yy, yz], [-xz.T, -yz.T, zz]])


def compressed_q(grid, layers, freq):
    """Q(i, j) for i in [0, Ny), j in [0, Nx) in the layout [Ny][Nx][6][Nz][Nz]."""
    out = np.empty((grid.ny, grid.nx, 6, grid.nz, grid.nz), dtype=np.complex128)
    for i in range(grid.ny):
        for j in range(grid.nx):
            out[i, j] = offset_blocks(grid, layers, freq, i, j)
    return out


def all_offsets(grid, layers, freq):
    """Q(i, j) for every signed offset, computed directly (no symmetry used):
    array [2Ny-1][2Nx-1][6][Nz][Nz] indexed by (i + Ny - 1, j + Nx - 1)."""
    ny, nx, nz = grid.ny, grid.nx, grid.nz
    out = np.empty((2 * ny - 1, 2 * nx - 1, 6, nz, nz), dtype=np.complex128)
    for i in range(-ny + 1, ny):
        for j in range(-nx + 1, nx):
            out[i + ny - 1, j + nx - 1] = offset_blocks(grid, layers, freq, i, j)
    return out
