"""Plain boundary-value solve of eq. (lmff) for one source point, used to pin the
oracle's closed-form fundamental functions.  Test code only.

In every piece of the line (layers, with the source layer split at z*) the solution
is a e^{-eta (z - top)} + b e^{-eta (bot - z)}; the half-spaces keep only the
decaying exponential.  The 2(L+1) unknowns follow from continuity of U and of
(1/gamma) U' at the interfaces, continuity of U and the jump -2 of U' at z*.
"""
import numpy as np

MU0 = 4e-7 * np.pi


def solve_U(layers, omega, lam, gamma, zs):
    d = list(layers.interfaces)
    sig = np.asarray(layers.sigma, dtype=np.complex128)
    L = len(d)
    eta = np.sqrt(lam ** 2 - 1j * omega * MU0 * sig)
    g = np.ones(L + 1, dtype=np.complex128) if gamma == "1" else sig.copy()
    s = int(np.searchsorted(np.asarray(d), zs, side="right"))
    # pieces: (top, bot, layer)
    bounds = [-np.inf] + d + [np.inf]
    pieces = []
    for m in range(L + 1):
        top, bot = bounds[m], bounds[m + 1]
        if m == s:
            pieces.append((top, zs, m))
            pieces.append((zs, bot, m))
        else:
            pieces.append((top, bot, m))
    # unknowns: (a, b) per piece; a multiplies e^{-eta(z-top)} (absent if top=-inf),
    # b multiplies e^{-eta(bot-z)} (absent if bot=+inf)
    idx = []
    n = 0
    for top, bot, m in pieces:
        ia = None if np.isinf(top) else n
        n += 0 if ia is None else 1
        ib = None if np.isinf(bot) else n
        n += 0 if ib is None else 1
        idx.append((ia, ib))

    def val_row(k, z, deriv):
        top, bot, m = pieces[k]
        e = eta[m]
        row = np.zeros(n, dtype=np.complex128)
        ia, ib = idx[k]
        if ia is not None:
            v = np.exp(-e * (z - top))
            row[ia] = -e * v if deriv else v
        if ib is not None:
            v = np.exp(-e * (bot - z))
            row[ib] = e * v if deriv else v
        return row

    A, rhs = [], []
    for k in range(len(pieces) - 1):
        zb = pieces[k][1]
        m1, m2 = pieces[k][2], pieces[k + 1][2]
        A.append(val_row(k, zb, False) - val_row(k + 1, zb, False)); rhs.append(0.0)
        if m1 == m2:   # the source point
            A.append(val_row(k + 1, zb, True) - val_row(k, zb, True)); rhs.append(-2.0)
        else:
            A.append(val_row(k, zb, True) / g[m1] - val_row(k + 1, zb, True) / g[m2]); rhs.append(0.0)
    coef = np.linalg.solve(np.array(A), np.array(rhs, dtype=np.complex128))

    def U(z):
        for k, (top, bot, m) in enumerate(pieces):
            if top <= z <= bot:
                return val_row(k, z, False) @ coef
        raise ValueError
    return U
