"""Pins for the assembled operator, the normal field and the solvers (oracle)."""
import numpy as np
import pytest

import workloads as W
from oracle import coefficients as C, normal, operator as O
from tests.oracle_cache import all_offsets_cached


@pytest.fixture(scope="module")
def small():
    m = W.small_model(nx=5, ny=4, nz=3, seed=11, freq=3.0)
    qa = all_offsets_cached(m)
    return m, qa


@pytest.fixture(scope="module")
def c1():
    m = W.config1()
    return m, all_offsets_cached(m)


def test_normal_field_half_space():
    sig = 0.02
    lay = W.Layers((0.0, 5000.0), (W.AIR_SIGMA, sig, sig))
    for f in (0.01, 1.0, 100.0):
        om = 2 * np.pi * f
        Z = normal.surface_impedance(lay, om)
        rho_a = abs(Z) ** 2 / (om * normal.MU0)
        assert abs(rho_a * sig - 1.0) < 1e-12
        assert abs(abs(np.degrees(np.angle(Z))) - 45.0) < 1e-9


def test_normal_field_ode_and_continuity():
    lay = W.Layers((0.0, 300.0, 800.0), (W.AIR_SIGMA, 0.01, 0.3, 0.002))
    om = 2 * np.pi * 2.0
    h = 0.05
    for z in (100.0, 500.0, 1500.0):
        m = int(np.searchsorted(np.asarray(lay.interfaces), z, side="right"))
        e = normal.field(lay, om, [z - h, z, z + h])
        d2 = (e[0] - 2 * e[1] + e[2]) / h ** 2
        assert abs(d2 + 1j * om * normal.MU0 * lay.sigma[m] * e[1]) < 1e-5 * abs(d2)
    for d in (300.0, 800.0):
        e = normal.field(lay, om, [d - 1e-7, d + 1e-7])
        assert abs(e[0] - e[1]) < 1e-8 * abs(e[0])
    e = normal.field(lay, om, [0.0, 1e-3])
    assert abs((e[1] - e[0]) / 1e-3 - 1j * om * normal.MU0) < 1e-4 * om * normal.MU0
    # the cell average equals the quadrature of the profile
    zz = np.linspace(300.0, 500.0, 20001)
    ee = normal.field(lay, om, zz)
    avg = np.trapezoid(ee, zz) / 200.0
    assert abs(normal.cell_average(lay, om, 300.0, 500.0) - avg) < 1e-7 * abs(avg)


def test_lateral_parities_lemma2(small):
    """Blocks computed independently at negative offsets obey (tensor_symm_2)."""
    m, qa = small
    ny, nx = m.grid.ny, m.grid.nx
    scale = np.abs(qa).max()
    for i in range(ny):
        for j in range(nx):
            q = qa[i + ny - 1, j + nx - 1]
            for b, (px, py) in enumerate(O.PARITY):
                assert np.abs(qa[-i + ny - 1, j + nx - 1, b] - py * q[b]).max() <= 1e-10 * scale
                assert np.abs(qa[i + ny - 1, -j + nx - 1, b] - px * q[b]).max() <= 1e-10 * scale
                assert np.abs(qa[-i + ny - 1, -j + nx - 1, b] - px * py * q[b]).max() <= 1e-10 * scale
    # odd parities force zeros on the axes
    assert np.abs(qa[ny - 1, :, 3]).max() <= 1e-10 * scale   # xy at i = 0
    assert np.abs(qa[:, nx - 1, 3]).max() <= 1e-10 * scale   # xy at j = 0
    assert np.abs(qa[:, nx - 1, 4]).max() <= 1e-10 * scale   # xz at j = 0
    assert np.abs(qa[ny - 1, :, 5]).max() <= 1e-10 * scale   # yz at i = 0


def test_vertical_symmetries_lemma1(small):
    """xx, yy, zz, xy blocks are symmetric in (z, z0) (eq. (matrix_symm))."""
    m, qa = small
    scale = np.abs(qa).max()
    for b in range(4):
        blk = qa[:, :, b]
        assert np.abs(blk - np.swapaxes(blk, -1, -2)).max() <= 1e-10 * scale


def test_reciprocity_and_contraction(small, c1):
    for mod, qa in (small, c1):
        B = O.dense_B(mod, qa)
        assert np.abs(B - B.T).max() <= 1e-11 * np.abs(B).max()
        nrm = O.contraction_norm(mod, B)
        assert nrm <= 1.0 + 1e-9, nrm


def test_fft_apply_equals_dense(small, c1):
    for mod, qa in (small, c1):
        g = mod.grid
        B = O.dense_B(mod, qa)
        A = O.dense_matrix(mod, B)
        q = qa[g.ny - 1:, g.nx - 1:]
        qt = O.full_spectrum_blocks(O.embed_spectrum(q))
        for seed in (1, 2):
            x = W.random_field((3, g.nz, g.ny, g.nx), seed)
            y = (A @ x.ravel()).reshape(x.shape)
            assert np.linalg.norm(O.fft_apply(mod, qt, x) - y) <= 1e-13 * np.linalg.norm(y) * 10
            yt = (A.T @ x.ravel()).reshape(x.shape)
            assert np.linalg.norm(O.fft_apply(mod, qt, x, transpose=True) - yt) <= 1e-12 * np.linalg.norm(yt)


def test_no_anomaly_gives_normal_field(small):
    m, qa = small
    sb = W.background_sigma(m.grid, m.layers)
    same = W.Model(m.name, m.grid, m.layers, np.broadcast_to(sb[:, None, None], m.sigma_a.shape).copy(),
                   m.freqs, m.pols)
    g = m.grid
    q = qa[g.ny - 1:, g.nx - 1:]
    qt = O.full_spectrum_blocks(O.embed_spectrum(q))
    b = normal.rhs_U0(same, m.freqs[0], "x")
    x, it, hist = O.gmres(lambda v: O.fft_apply(same, qt, v), b, tol=1e-12)
    assert it == 1 and np.linalg.norm(x - b) <= 1e-14 * np.linalg.norm(b)


def test_lu_equals_gmres_and_contraction_rate(c1):
    m, qa = c1
    g = m.grid
    B = O.dense_B(m, qa)
    A = O.dense_matrix(m, B)
    q = qa[g.ny - 1:, g.nx - 1:]
    qt = O.full_spectrum_blocks(O.embed_spectrum(q))
    b = normal.rhs_U0(m, m.freqs[0], "x")
    u_lu = np.linalg.solve(A, b.ravel()).reshape(b.shape)
    u, it, hist = O.gmres(lambda v: O.fft_apply(m, qt, v), b, tol=1e-12, m=30)
    assert np.linalg.norm(u - u_lu) <= 1e-10 * np.linalg.norm(u_lu)
    res = np.linalg.norm(b - O.fft_apply(m, qt, u)) / np.linalg.norm(b)
    assert res <= 1e-11


def test_in_cell_field_without_anomaly_is_the_normal_field():
    """sigma_a = sigma_b: U = U^0 = s <E^N>, so E = U / a must be the cell average of the
    1-D normal field itself (a = Re sigma_b / s = s)."""
    m0 = W.small_model(nx=4, ny=3, nz=4, seed=7, freq=2.0)
    sb = W.background_sigma(m0.grid, m0.layers)
    m = W.Model(m0.name, m0.grid, m0.layers, np.broadcast_to(sb[:, None, None], m0.sigma_a.shape).copy(),
                m0.freqs, m0.pols)
    ze = m.grid.z_edges_array()
    om = 2 * np.pi * m.freqs[0]
    avg = np.array([normal.cell_average(m.layers, om, ze[k], ze[k + 1]) for k in range(m.grid.nz)])
    for pol, c in (("x", 0), ("y", 1)):
        E = O.in_cell_field(m, normal.rhs_U0(m, m.freqs[0], pol))
        ref = np.zeros_like(E)
        ref[c] = avg[:, None, None]
        assert np.abs(E - ref).max() <= 1e-13 * np.abs(avg).max()


def test_in_cell_field_gives_the_scattering_current():
    """(sigma_a - sigma_b) E = 2 s gamma U: the current of (APR_lab) written with the
    in-cell field equals the one written with gamma of (slae_matricies)."""
    m = W.small_model(nx=5, ny=4, nz=3, seed=11, freq=3.0)
    U = W.random_field((2, 3, m.grid.nz, m.grid.ny, m.grid.nx), 5)
    gamma, s, V = O.diagonals(m)
    sb = W.background_sigma(m.grid, m.layers)
    J1 = (m.sigma_a - sb[:, None, None]) * O.in_cell_field(m, U)
    J2 = 2.0 * s[:, None, None] * gamma * U
    assert np.abs(gamma).max() > 0.1
    assert np.abs(J1 - J2).max() <= 1e-13 * np.abs(J2).max()

