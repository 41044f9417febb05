"""Fundamental functions of the layered medium and the vertical integrals.

Test infrastructure (see ``oracle/__init__``).  Paper: Appendix B.

U_gamma(z, z*, lambda), gamma in {1, sigma}, is the unique solution of eq. (lmff):
U'' - eta_m^2 U = 0 inside layer m, U continuous, (1/gamma) U' continuous at the
interfaces, [U]_{z*} = 0, [U']_{z*} = -2, decay at +-infinity, with
eta_m^2 = lambda^2 - k_m^2 and k_m^2 = i omega mu0 sigma_m.

It is built with the recursions (pq_req) for p_m, q_m, the amplitudes (A_rs),
and evaluated in the overflow-free form (UU2): every exponential is grouped so
that its exponent has a non-positive real part at the point of evaluation.

Readings of the paper used here:
* (UU2), second branch: the third exponent is read as e^{-(eta_r z_r - eta_s z_s)},
  the mirror of the first branch.
* (U_explicit), second branch (field point below the source point): the
  amplitude is A_{r,s} with r the layer of the field point, i.e. by the last line
  of (A_rs) A^sigma_{r,s} = (sigma_r / sigma_s) A^sigma_{s,r}.  With A_{s,r} the
  condition on (1/sigma) U' at an interface between source and field would fail;
  the substitution test in tests/test_oracle_layered.py pins this.
* V3..V5 of (Ver_Int) are evaluated with the fundamental theorem of calculus on
  the nested integrals (cell-face values).  V3 so obtained contains the delta
  of d/dz d/dz* U at z = z*; see ``coefficients`` for how it is used.

Pins: substitution into (lmff) (ODE residual, interface and jump conditions),
the homogeneous whole-space closed form U = e^{-eta|z-z*|}/eta, and a brute-force
quadrature of the vertical integrals (tests/test_oracle_layered.py).
"""
from __future__ import annotations

import numpy as np

MU0 = 4e-7 * np.pi


def _phi_ab(x):
    """(x - 1 + e^{-x}) / x^2, stable for small |x|."""
    x = np.asarray(x, dtype=np.complex128)
    out = np.empty_like(x)
    small = np.abs(x) < 0.05
    xs = x[small]
    # series sum_{k>=2} (-1)^k x^{k-2} / k!
    s = np.zeros_like(xs)
    term = np.full_like(xs, 0.5)
    for k in range(2, 14):
        s = s + term
        term = term * (-xs) / (k + 1)
    out[small] = s
    xl = x[~small]
    out[~small] = (xl - 1.0 + np.exp(-xl)) / xl ** 2
    return out


def _psi_ab(x):
    """(1 - e^{-x}(1 + x)) / x^2, stable for small |x|."""
    x = np.asarray(x, dtype=np.complex128)
    out = np.empty_like(x)
    small = np.abs(x) < 0.05
    xs = x[small]
    # 1 - e^{-x}(1+x) = sum_{k>=2} (-1)^k (k-1) x^k / k!
    s = np.zeros_like(xs)
    fact = 2.0
    pw = np.ones_like(xs)
    for k in range(2, 16):
        s = s + ((-1) ** k) * (k - 1) * pw / fact
        pw = pw * xs
        fact *= (k + 1)
    out[small] = s
    xl = x[~small]
    out[~small] = (1.0 - np.exp(-xl) * (1.0 + xl)) / xl ** 2
    return out


def _int_exp(a, x1, x2):
    """Integral of e^{a x} over [x1, x2] as (reference point, factor): the integral is
    e^{a * ref} * factor, with ref the end point where Re(a x) is largest."""
    h = x2 - x1
    pos = a.real >= 0
    ref = np.where(pos, x2, x1)
    with np.errstate(invalid="ignore", divide="ignore", over="ignore"):
        f = np.where(pos, -np.expm1(-a * h) / a, np.expm1(a * h) / a)
    f = np.where(np.abs(a) * h < 1e-300, h, f)
    return ref, f


class Spectrum:
    """p, q, A and the transfer factors of (pq_req), (A_rs) at an array of lambda."""

    def __init__(self, layers, omega, lam, gamma):
        d = np.asarray(layers.interfaces, dtype=np.float64)
        sig = np.asarray(layers.sigma, dtype=np.complex128)
        lam = np.asarray(lam, dtype=np.float64)
        L = len(d)
        self.L = L
        self.gamma = gamma
        self.sig = sig
        # d_m for m = 0..L+1 with d_0 = d_1 and d_{L+1} = d_L
        self.d = np.concatenate([[d[0]], d, [d[-1]]])
        l = np.zeros(L + 1)
        l[1:L] = np.diff(d)
        self.l = l
        k2 = 1j * omega * MU0 * sig
        eta = np.sqrt(lam[:, None] ** 2 - k2[None, :])
        self.eta = eta
        n = lam.shape[0]
        if gamma == "1":
            alpha = np.ones(L, dtype=np.complex128)           # alpha_m, m = 0..L-1
            beta = np.ones(L + 1, dtype=np.complex128)        # beta_m, m = 1..L (index 0 unused)
        else:
            alpha = sig[1:] / sig[:-1]
            beta = np.concatenate([[1.0], sig[:-1] / sig[1:]])
        p = np.zeros((n, L + 1), dtype=np.complex128)
        for m in range(0, L):
            e = p[:, m] * np.exp(-2.0 * eta[:, m] * l[m])
            X = (e - 1.0) / (e + 1.0)
            ra = alpha[m] * eta[:, m] / eta[:, m + 1]
            p[:, m + 1] = (1.0 + ra * X) / (1.0 - ra * X)
        q = np.zeros((n, L + 1), dtype=np.complex128)
        for m in range(L, 0, -1):
            e = q[:, m] * np.exp(-2.0 * eta[:, m] * l[m])
            Y = (e - 1.0) / (e + 1.0)
            rb = beta[m] * eta[:, m] / eta[:, m - 1]
            q[:, m - 1] = (1.0 + rb * Y) / (1.0 - rb * Y)
        self.p, self.q = p, q
        self.Ann = 1.0 / (eta * (1.0 - p * q * np.exp(-2.0 * eta * l[None, :])))
        # transfer factor of Q_m without its exponential e^{(eta_{m+1}-eta_m) d_{m+1}}
        t = np.ones((n, L + 1), dtype=np.complex128)
        for m in range(0, L):
            t[:, m] = (1.0 + p[:, m + 1]) / (1.0 + p[:, m] * np.exp(-2.0 * eta[:, m] * l[m]))
        self.t = t

    def terms(self, r, s, below):
        """Exponential terms of U(z, z*) for z in layer r, z* in layer s.

        below=False: z <= z* (requires r <= s);  below=True: z > z* (requires r >= s).
        Returns a list of (coef, a_z, a_zs, const) with U = sum coef*exp(a_z z + a_zs z* + const).
        """
        eta, d, l, p, q = self.eta, self.d, self.l, self.p, self.q
        if not below:
            up, lo = r, s          # upper point in layer up (the field point)
        else:
            up, lo = s, r          # upper point is the source point
        amp = self.Ann[:, lo].copy()
        for m in range(up, lo):
            amp = amp * self.t[:, m]
        if below and self.gamma == "sigma" and r != s:
            amp = amp * (self.sig[r] / self.sig[s])
        eu, el = eta[:, up], eta[:, lo]
        if up == lo:
            c0 = np.zeros_like(eu)
        else:
            c0 = -eu * d[up + 1] + el * d[lo]
            for m in range(up + 1, lo):
                c0 = c0 - eta[:, m] * l[m]
        pu, ql = p[:, up], q[:, lo]
        # upper factor (1 + p_up e^{-2 eta_up (x_up - d_up)}), lower (1 + q_lo e^{-2 eta_lo (d_{lo+1} - x_lo)})
        # tags: "d" depends on x_lo - x_up and decays, "s" separable, "g" depends on
        # x_lo - x_up and grows with it.  Terms whose coefficient vanishes identically
        # (p_0 = 0 in the air, q_L = 0 in the basement) are left out: their exponent
        # need not be bounded there.
        base = [(amp, eu, -el, c0, "d")]
        if up >= 1:
            base.append((amp * pu, -eu, -el, c0 + 2 * eu * d[up], "s"))
        if lo < self.L:
            base.append((amp * ql, eu, el, c0 - 2 * el * d[lo + 1], "s"))
        if up >= 1 and lo < self.L:
            base.append((amp * pu * ql, -eu, el, c0 + 2 * eu * d[up] - 2 * el * d[lo + 1], "g"))
        if not below:
            return base                      # x_up = z, x_lo = z*
        return [(c, b, a, k, g) for (c, a, b, k, g) in base]   # x_up = z*, x_lo = z


class StaticSpectrum:
    """The large-lambda (quasi-static) limit of U_sigma used as the subtracted part.

    Same layer r:  e^{-lam|z-z*|}/lam + P_top e^{-lam(z+z*-2 d_r)}/lam + P_bot e^{-lam(2 d_{r+1}-z-z*)}/lam
    Adjacent layers (field r, source s):  T_rs e^{-lam|z-z*|}/lam
    with P_top = (s_{r-1}-s_r)/(s_{r-1}+s_r), P_bot = (s_{r+1}-s_r)/(s_{r+1}+s_r),
    T_rs = 2 s_r/(s_r+s_s): the lambda -> infinity limits of p_r, q_r and of the
    transfer amplitude for gamma = sigma in (pq_req), (A_rs).
    """

    def __init__(self, layers, lam):
        d = np.asarray(layers.interfaces, dtype=np.float64)
        self.sig = np.asarray(layers.sigma, dtype=np.complex128)
        self.L = len(d)
        self.d = np.concatenate([[d[0]], d, [d[-1]]])
        self.lam = np.asarray(lam, dtype=np.float64).astype(np.complex128)

    def coefs(self, r, s):
        sg = self.sig
        if r == s:
            pt = (sg[r - 1] - sg[r]) / (sg[r - 1] + sg[r]) if r >= 1 else 0.0
            pb = (sg[r + 1] - sg[r]) / (sg[r + 1] + sg[r]) if r < self.L else 0.0
            return 1.0, pt, pb
        if abs(r - s) == 1:
            return 2 * sg[r] / (sg[r] + sg[s]), 0.0, 0.0
        return 0.0, 0.0, 0.0

    def terms(self, r, s, below):
        lam = self.lam
        c, pt, pb = self.coefs(r, s)
        d = self.d
        inv = 1.0 / lam
        zero = np.zeros_like(lam)
        if c == 0.0:
            return []
        out = [(c * inv, -lam, lam, zero, "d") if below else (c * inv, lam, -lam, zero, "d")]
        if r == s and pt != 0.0:
            out.append((pt * inv, -lam, -lam, 2 * lam * d[r], "s"))
        if r == s and pb != 0.0:
            out.append((pb * inv, lam, lam, -2 * lam * d[r + 1], "s"))
        return out


def _eval_terms(terms, z, zs):
    acc = 0.0
    for c, a, b, k, _ in terms:
        acc = acc + c * np.exp(a * z + b * zs + k)
    return acc


def _F(terms, z0, w1, w2, deriv=False):
    """int_{w1}^{w2} U(z0, z*) dz*  (or of dU/dz when deriv)."""
    acc = 0.0
    for c, a, b, k, _ in terms:
        wr, vb = _int_exp(b, w1, w2)
        v = c * np.exp(a * z0 + b * wr + k) * vb
        acc = acc + (a * v if deriv else v)
    return acc


def _DD_disjoint(terms, z1, z2, w1, w2):
    acc = 0.0
    for c, a, b, k, _ in terms:
        zr, va = _int_exp(a, z1, z2)
        wr, vb = _int_exp(b, w1, w2)
        acc = acc + c * np.exp(a * zr + b * wr + k) * va * vb
    return acc


def _DD_self(terms, z1, z2):
    """Double integral over the square [z1,z2]^2 for a pair within one cell.

    ``terms`` are those of the branch z <= z*.  A term tagged "d" is
    e^{k} e^{-eta (z*-z)} there and e^{k} e^{-eta |z-z*|} on the whole square;
    a term tagged "g" is e^{k} e^{+eta |z-z*|}; "s" terms are the same on both
    branches and separable."""
    h = z2 - z1
    out = 0.0
    for c, a, b, k, tag in terms:
        if tag == "d":
            eta = a
            out = out + c * np.exp(k) * 2.0 * h * h * _phi_ab(eta * h)
        elif tag == "g":
            eta = b
            out = out + c * np.exp(k + eta * h) * 2.0 * h * h * _psi_ab(eta * h)
        else:
            zr, va = _int_exp(a, z1, z2)
            wr, vb = _int_exp(b, z1, z2)
            out = out + c * np.exp(a * zr + b * wr + k) * va * vb
    return out


def pair_quantities(spec, z1, z2, r, w1, w2, s):
    """DD = int int U, F(z1), F(z2), F_z(z1), F_z(z2) and U at the four corners for the
    field cell [z1,z2] (layer r) and the source cell [w1,w2] (layer s)."""
    if z2 <= w1:            # field cell above the source cell
        t = spec.terms(r, s, False)
        DD = _DD_disjoint(t, z1, z2, w1, w2)
        F1, F2 = _F(t, z1, w1, w2), _F(t, z2, w1, w2)
        Fz1, Fz2 = _F(t, z1, w1, w2, True), _F(t, z2, w1, w2, True)
        corners = [_eval_terms(t, z, w) for z, w in ((z1, w1), (z1, w2), (z2, w1), (z2, w2))]
    elif z1 >= w2:          # field cell below the source cell
        t = spec.terms(r, s, True)
        DD = _DD_disjoint(t, z1, z2, w1, w2)
        F1, F2 = _F(t, z1, w1, w2), _F(t, z2, w1, w2)
        Fz1, Fz2 = _F(t, z1, w1, w2, True), _F(t, z2, w1, w2, True)
        corners = [_eval_terms(t, z, w) for z, w in ((z1, w1), (z1, w2), (z2, w1), (z2, w2))]
    else:
        assert z1 == w1 and z2 == w2 and r == s, "cells overlap without coinciding"
        ta = spec.terms(r, s, False)   # z <= z*
        tb = spec.terms(r, s, True)    # z >  z*
        DD = _DD_self(ta, z1, z2)
        F1, F2 = _F(ta, z1, w1, w2), _F(tb, z2, w1, w2)
        Fz1, Fz2 = _F(ta, z1, w1, w2, True), _F(tb, z2, w1, w2, True)
        corners = [_eval_terms(ta, z1, w1), _eval_terms(ta, z1, w2),
                   _eval_terms(tb, z2, w1), _eval_terms(ta, z2, w2)]
    return dict(DD=DD, F1=F1, F2=F2, Fz1=Fz1, Fz2=Fz2, U11=corners[0], U12=corners[1],
                U21=corners[2], U22=corners[3])


def cell_layers(layers, z_edges):
    """Layer index of every z-cell; raises if a cell straddles an interface."""
    d = np.asarray(layers.interfaces, dtype=np.float64)
    out = []
    for k in range(len(z_edges) - 1):
        a, b = z_edges[k], z_edges[k + 1]
        ra = int(np.searchsorted(d, a, side="right"))
        rb = int(np.searchsorted(d, b, side="left"))
        if ra != rb:
            raise ValueError(f"cell [{a}, {b}] straddles a layer interface")
        out.append(ra)
    return np.array(out, dtype=int)


def vertical_integrals(layers, omega, z_edges, lam, static=False):
    """V1..V5 of (Ver_Int) for every pair (field cell a, source cell b).

    Returns a dict of complex arrays of shape (n_lam, Nz, Nz):
      V1 = i w mu0 int int U_1,  V2 = i w mu0 int int U_sigma,
      V3w = -(1/sigma_a) [U(z2,w2) - U(z2,w1) - U(z1,w2) + U(z1,w1)]      (U = U_sigma)
      V4 = (1/sigma_a) [F(z2) - F(z1)],  V5 = (1/sigma_a) [F_z(z2) - F_z(z1)],
    with sigma_a the background conductivity of the field cell.
    ``static=True`` evaluates the same quantities for the quasi-static U_sigma of
    StaticSpectrum (V1, V2 are then omitted).
    """
    z_edges = np.asarray(z_edges, dtype=np.float64)
    nz = len(z_edges) - 1
    lay = cell_layers(layers, z_edges)
    sig = np.asarray(layers.sigma, dtype=np.complex128)
    lam = np.asarray(lam, dtype=np.float64)
    n = lam.shape[0]
    if static:
        specs = {"sigma": StaticSpectrum(layers, lam)}
    else:
        specs = {"1": Spectrum(layers, omega, lam, "1"), "sigma": Spectrum(layers, omega, lam, "sigma")}
    out = {k: np.zeros((n, nz, nz), dtype=np.complex128) for k in ("V1", "V2", "V3w", "V4", "V5")}
    iwm = 1j * omega * MU0
    for a in range(nz):
        z1, z2, r = z_edges[a], z_edges[a + 1], lay[a]
        for b in range(nz):
            w1, w2, s = z_edges[b], z_edges[b + 1], lay[b]
            qs = pair_quantities(specs["sigma"], z1, z2, r, w1, w2, s)
            inv = 1.0 / sig[r]
            out["V3w"][:, a, b] = -inv * (qs["U22"] - qs["U21"] - qs["U12"] + qs["U11"])
            out["V4"][:, a, b] = inv * (qs["F2"] - qs["F1"])
            out["V5"][:, a, b] = inv * (qs["Fz2"] - qs["Fz1"])
            if not static:
                out["V2"][:, a, b] = iwm * qs["DD"]
                q1 = pair_quantities(specs["1"], z1, z2, r, w1, w2, s)
                out["V1"][:, a, b] = iwm * q1["DD"]
    return out


def evaluate_U(layers, omega, lam, gamma, z, zs, r=None, s=None):
    """U_gamma(z, z*, lambda) at scalar points (used by the substitution tests).

    r, s: layers of z and z*; by default the layer below when a point lies on an
    interface.  U_sigma is discontinuous in z* across an interface (the factor
    sigma_r/sigma_s of (A_rs)), so the layer matters there."""
    d = np.asarray(layers.interfaces, dtype=np.float64)
    r = int(np.searchsorted(d, z, side="right")) if r is None else r
    s = int(np.searchsorted(d, zs, side="right")) if s is None else s
    spec = Spectrum(layers, omega, np.atleast_1d(lam), gamma)
    t = spec.terms(r, s, z > zs)
    return _eval_terms(t, z, zs)


def evaluate_dU(layers, omega, lam, gamma, z, zs, r=None, s=None):
    """dU/dz at (z, z*) from the analytic form (one-sided inside the layer of z)."""
    d = np.asarray(layers.interfaces, dtype=np.float64)
    r = int(np.searchsorted(d, z, side="right")) if r is None else r
    s = int(np.searchsorted(d, zs, side="right")) if s is None else s
    spec = Spectrum(layers, omega, np.atleast_1d(lam), gamma)
    t = spec.terms(r, s, z > zs)
    acc = 0.0
    for c, a, b, k, _ in t:
        acc = acc + a * c * np.exp(a * z + b * zs + k)
    return acc
