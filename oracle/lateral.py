"""Lateral (horizontal) cell-to-cell kernels of the Hankel integrals, eq. (Hor_Int).

Test infrastructure (see ``oracle/__init__``).  Paper: Appendix A, eq. (Hor_Int);
Appendix C, eq. (g_eint), (transf).

For two cells with equal lateral sizes hx, hy and lateral offset D = (Dx, Dy)
(field cell minus source cell), the four-fold lateral integral of J0(lambda rho)
is the function of lambda

  K_J(lam; D) = int_{S_n} int_{S_m} J0(lam rho) dS_m dS_n,

the quantity lambda^{-4} K(R lambda; p, q, phi) of eq. (transf).  The lateral
derivatives of (Hor_Int) act on the offset:

  K_xx = d2 K_J/dDx2,  K_yy = d2 K_J/dDy2,  K_xy = d2 K_J/dDx dDy,
  K_x = d K_J/dDx,     K_y = d K_J/dDy.

They are evaluated through the two-dimensional Fourier representation of J0:
J0(lam rho) = (1/2pi) int_0^{2pi} exp(i lam (x cos t + y sin t)) dt, which turns the
rectangles into the transforms T_h(k) = h^2 sinc^2(k h / 2) of their
autocorrelation (tent) functions:

  K_J = (2/pi) int_0^{pi/2} T_hx(lam c) T_hy(lam s) cos(lam c Dx) cos(lam s Dy) dt,

c = cos t, s = sin t, and the derivatives bring down -k_x^2, -k_y^2, k_x k_y
(sin sin), -k_x (sin cos), -k_y (cos sin).  The integrand is an analytic
periodic function of t, so the trapezoidal rule converges exponentially once the
number of nodes exceeds its bandwidth lam (|Dx| + |Dy| + hx + hy).

Pins: K_J(0) = hx^2 hy^2; direct spatial quadrature of the J0 integrals; finite
differences of K_J in Dx, Dy; and int_0^inf K_J e^{-lam a} dlam equal to the
closed-form static lateral integral (tests/test_oracle_lateral.py).
"""
from __future__ import annotations

import numpy as np


def _tent_hat(k, h):
    return h * h * np.sinc(k * h / (2.0 * np.pi)) ** 2


def n_theta(lam, Dx, Dy, hx, hy):
    band = lam * (abs(Dx) + abs(Dy) + hx + hy)
    return (np.ceil(0.32 * band) + 24).astype(int)


def lateral_kernels(lam, Dx, Dy, hx, hy, block=64):
    """Dict of K_J, K_xx, K_yy, K_xy, K_x, K_y at the lambda array ``lam``."""
    lam = np.asarray(lam, dtype=np.float64)
    order = np.argsort(lam)
    out = {k: np.zeros(lam.shape[0]) for k in ("J", "xx", "yy", "xy", "x", "y")}
    nt_all = n_theta(lam, Dx, Dy, hx, hy)
    for s0 in range(0, lam.shape[0], block):
        idx = order[s0:s0 + block]
        nt = int(nt_all[idx].max())
        t = np.linspace(0.0, 0.5 * np.pi, nt + 1)
        w = np.full(nt + 1, 1.0 / nt)
        w[0] *= 0.5
        w[-1] *= 0.5
        L = lam[idx][:, None]
        kx = L * np.cos(t)[None, :]
        ky = L * np.sin(t)[None, :]
        base = _tent_hat(kx, hx) * _tent_hat(ky, hy) * w[None, :]
        cx, sx = np.cos(kx * Dx), np.sin(kx * Dx)
        cy, sy = np.cos(ky * Dy), np.sin(ky * Dy)
        bcc = base * cx * cy
        out["J"][idx] = bcc.sum(1)
        out["xx"][idx] = -(kx * kx * bcc).sum(1)
        out["yy"][idx] = -(ky * ky * bcc).sum(1)
        out["xy"][idx] = (kx * ky * base * sx * sy).sum(1)
        out["x"][idx] = -(kx * base * sx * cy).sum(1)
        out["y"][idx] = -(ky * base * cx * sy).sum(1)
    return out
