"""Pins of the oracle's solver and discretisation against properties the paper fixes.

* GMRES rate (Sect. 2.1-2.2): A = I - K Gamma with ||K|| <= 1 in the V-weighted norm
  (the contraction of the modified operator, eq. (Grmod)) and |gamma| <= q < 1, so
  p(A) = (I - A)^m = (K Gamma)^m is admissible in every restart cycle of GMRES(m):
  ||r_{j+1}||_2 <= c q^m ||r_j||_2 with c = sqrt(max V / min V) (c = 1 on a uniform
  grid).  Each cycle's residual must also be the minimum over its Krylov space,
  computed here by brute force from the dense matrix (a plain least-squares problem).
* Discretisation (Sect. 2.2, after eq. (pr_op)): the Galerkin solution converges
  to the field with the first order of the cell diameter d.  Halving d twice on a
  cube (1, 2, 4 cells per side; oracle coefficients, dense LU), the L2 distance
  between successive solutions must shrink: by a factor of at least 1.5 for the
  field (measured 1.68; the asymptotic factor of a first-order method is 2, three
  levels are pre-asymptotic) and of at least 1.25 for its scattered part E - <E^N>
  (measured 1.40: the scattered field is singular at the edges of the anomaly, so
  it converges more slowly on coarse grids).
"""
import numpy as np
import pytest

import workloads as W
from oracle import coefficients, normal, operator as O
from tests.oracle_cache import all_offsets_cached


def _check_rate(m, qa, restart, cycles):
    g = m.grid
    A = O.dense_matrix(m, O.dense_B(m, qa))
    gamma, s, V = O.diagonals(m)
    q = float(np.abs(gamma).max())
    assert q < 1.0
    c = float(np.sqrt(V.max() / V.min()))
    b = normal.rhs_U0(m, m.freqs[0], "x")
    nb = np.linalg.norm(b)
    x = np.zeros_like(b)
    for j in range(cycles):
        r0 = (b.ravel() - A @ x.ravel())
        x1, it, hist = O.gmres(lambda v: (A @ v.ravel()).reshape(v.shape), b, tol=1e-30, m=restart,
                               max_iter=restart, x0=x)
        r1 = b.ravel() - A @ x1.ravel()
        # rate bound of the contracting operator
        assert np.linalg.norm(r1) <= c * q ** restart * np.linalg.norm(r0) * (1 + 1e-12), (j, q)
        # optimality: the minimum of ||r0 - A Z y|| over the Krylov space span(r0, A r0, ...)
        Z = np.empty((r0.size, restart), dtype=np.complex128)
        Z[:, 0] = r0 / np.linalg.norm(r0)
        for k in range(1, restart):
            w = A @ Z[:, k - 1]
            w -= Z[:, :k] @ (Z[:, :k].conj().T @ w)
            w -= Z[:, :k] @ (Z[:, :k].conj().T @ w)
            Z[:, k] = w / np.linalg.norm(w)
        y = np.linalg.lstsq(A @ Z, r0, rcond=None)[0]
        best = np.linalg.norm(r0 - A @ (Z @ y))
        assert abs(np.linalg.norm(r1) - best) <= 1e-9 * np.linalg.norm(r0) + 1e-12 * nb, (j, best)
        x = x1


def test_gmres_rate_bound_c1():
    m = W.config1()
    _check_rate(m, all_offsets_cached(m), restart=3, cycles=5)


def test_gmres_rate_bound_small_model():
    m = W.small_model(nx=5, ny=4, nz=3, seed=11, freq=3.0)
    _check_rate(m, all_offsets_cached(m), restart=2, cycles=6)


def _cube_solution(n, sig_b, sig_a, f, side):
    lay = W.Layers((0.0,), (W.AIR_SIGMA, sig_b))
    h = side / n
    g = W.Grid(n, n, n, h, h, tuple(h * k for k in range(n + 1)))
    m = W.Model(f"cube{n}", g, lay, np.full((n, n, n), sig_a, dtype=np.complex128), (f,), ("x",))
    A = O.dense_matrix(m, O.dense_B(m, all_offsets_cached(m)))
    b = normal.rhs_U0(m, f, "x")
    U = np.linalg.solve(A, b.ravel()).reshape(b.shape)
    E = O.in_cell_field(m, U)
    om = 2 * np.pi * f
    en = np.array([normal.cell_average(lay, om, g.z_edges[k], g.z_edges[k + 1]) for k in range(n)])
    Es = E.copy()
    Es[0] -= en[:, None, None]
    return E, Es


def test_first_order_convergence_in_cell_size():
    side, sig_b, sig_a, f = 200.0, 0.01, 0.02, 1000.0
    sols = {n: _cube_solution(n, sig_b, sig_a, f, side) for n in (1, 2, 4)}

    def up(a, k):
        return a.repeat(k, axis=1).repeat(k, axis=2).repeat(k, axis=3)

    for part, factor in ((0, 1.5), (1, 1.25)):  # total field, scattered field
        d = []
        for a, bb in ((1, 2), (2, 4)):
            hf = side / bb
            d.append(np.sqrt(np.sum(np.abs(sols[bb][part] - up(sols[a][part], bb // a)) ** 2) * hf ** 3))
        assert d[1] < d[0] / factor, (part, d)
