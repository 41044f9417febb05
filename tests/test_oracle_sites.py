"""Pins of the oracle's field recovery at arbitrary sites (eq. (APR_lab)) and of the MT
maps: at cell centres the site operator is the cell-centred one; a site moved by a
whole cell sees the same kernels one cell further; without an anomaly the apparent
resistivity of a half-space is 1/sigma at 45 degrees."""
import numpy as np

import workloads as W
from oracle import normal, receivers as RC


def _grid():
    layers = W.Layers((0.0, 140.0), (1e-9, 0.02, 0.005))
    grid = W.uniform_grid(3, 2, 2, 50.0, z0=40.0)
    return grid, layers


def test_site_operator_at_cell_centres_is_the_cell_operator():
    grid, layers = _grid()
    cells = [(0, 0), (1, 2), (0, 1)]  # (iy, ix)
    G1 = RC.receiver_operator(grid, layers, 2.0, 0.0, cells)
    sites = [((ix + 0.5) * grid.hx, (iy + 0.5) * grid.hy) for iy, ix in cells]
    G2 = RC.receiver_operator_sites(grid, layers, 2.0, 0.0, sites)
    assert np.max(np.abs(G1 - G2)) <= 1e-14 * np.max(np.abs(G1))


def test_site_kernels_translate_with_the_grid():
    """Moving the site by one cell in x and the cells with it leaves every kernel
    unchanged: the kernels depend on the offset site - cell only."""
    grid, layers = _grid()
    x, y = 0.37 * grid.hx, 1.21 * grid.hy
    G = RC.receiver_operator_sites(grid, layers, 2.0, 0.0, [(x, y), (x + grid.hx, y)])
    g0 = G[0].reshape(4, 3, grid.nz, grid.ny, grid.nx)
    g1 = G[1].reshape(4, 3, grid.nz, grid.ny, grid.nx)
    assert np.max(np.abs(g0[..., :-1] - g1[..., 1:])) <= 1e-13 * np.max(np.abs(g0))


def test_apparent_resistivity_of_a_half_space():
    sig = 0.01
    layers = W.Layers((0.0,), (1e-9, sig))
    grid = W.uniform_grid(2, 2, 2, 100.0, z0=100.0)
    sb = W.background_sigma(grid, layers)
    m = W.Model("hs", grid, layers, np.broadcast_to(sb[:, None, None], (2, 2, 2)).astype(np.complex128).copy(),
                (1.0,), ("x", "y"))
    G = RC.receiver_operator_sites(grid, layers, 1.0, 0.0, [(37.0, 151.0), (200.0, 0.0)])
    U = np.stack([normal.rhs_U0(m, 1.0, "x"), normal.rhs_U0(m, 1.0, "y")])
    rho, ph = RC.apparent(RC.impedance(RC.fields(m, 1.0, U, G, 0.0)), 1.0)
    for r in range(2):
        assert abs(rho[r, 0, 1] * sig - 1.0) < 1e-9 and abs(rho[r, 1, 0] * sig - 1.0) < 1e-9
        assert abs(abs(ph[r, 0, 1]) - 45.0) < 1e-7 and abs(abs(ph[r, 1, 0]) - 135.0) < 1e-7
