"""Field recovery at arbitrary sites (eq. (APR_lab)) and the MT maps on the GPU,
through the C ABI, against the oracle (oracle/receivers.py): sites at cell centres
against the cell-centred receivers, sites anywhere against the oracle's dense site
operator, the adjoint of the site operator by the bilinear identity, and the apparent
resistivity and phase against their definition."""
import numpy as np
import pytest

import workloads as W
from oracle import receivers as RC
from tests.gpu_support import need_gpu, to_dev, to_host, torch

pytestmark = pytest.mark.gpu


def _model(shape, seed=3):
    nx, ny, nz = shape
    layers = W.Layers((0.0, 140.0), (1e-9, 0.02, 0.005))
    grid = W.uniform_grid(nx, ny, nz, 50.0, z0=40.0)
    sb = W.background_sigma(grid, layers)
    rng = np.random.default_rng(seed)
    sa = np.broadcast_to(sb[:, None, None], (nz, ny, nx)).astype(np.complex128).copy()
    mask = rng.random((nz, ny, nx)) < 0.6
    sa[mask] = 10 ** rng.uniform(-2, 0, mask.sum())
    return W.Model("sites", grid, layers, sa, (2.0,), ("x", "y"))


def _ctx(m):
    from paper_1512_06126_gb300 import build, ie
    build.build()
    return ie.Context(m.grid, m.layers, m.sigma_a, m.freqs, None, max_rhs=2)


def _fields(ctx, U, n_rec):
    ud = to_dev(U)
    f1 = torch.empty((2, n_rec, 4), dtype=torch.complex128, device="cuda")
    f0 = torch.empty_like(f1)
    ctx.receiver_fields(0, ud.data_ptr(), 2, (0, 1), f1.data_ptr())
    ctx.receiver_fields(0, torch.zeros_like(ud).data_ptr(), 2, (0, 1), f0.data_ptr())
    return to_host(f1), to_host(f0)


def test_sites_at_cell_centres_match_cell_receivers():
    need_gpu()
    m = _model((7, 5, 3))
    g = m.grid
    ctx = _ctx(m)
    cells = [(0, 0), (6, 4), (3, 2), (1, 4)]  # (ix, iy)
    U = W.random_field((2, 3, g.nz, g.ny, g.nx), 17)
    ctx.set_receivers([c[0] for c in cells], [c[1] for c in cells], 0.0)
    fa, _ = _fields(ctx, U, len(cells))
    ctx.set_receivers_xy([(c[0] + 0.5) * g.hx for c in cells], [(c[1] + 0.5) * g.hy for c in cells], 0.0)
    fb, _ = _fields(ctx, U, len(cells))
    assert np.max(np.abs(fa - fb)) <= 1e-10 * np.max(np.abs(fa))
    ctx.close()


def test_site_fields_against_oracle():
    """Sites off the cell centres (two sharing a sub-cell position, one on the grid's
    edge, one at a corner), scattered fields against the oracle's dense site operator."""
    need_gpu()
    m = _model((7, 5, 3), seed=5)
    g = m.grid
    ctx = _ctx(m)
    sites = [(30.0, 60.0), (80.0, 110.0), (0.0, 137.5), (350.0, 250.0), (212.3, 41.9)]
    ctx.set_receivers_xy([s[0] for s in sites], [s[1] for s in sites], 0.0)
    G = RC.receiver_operator_sites(g, m.layers, 2.0, 0.0, sites)
    U = W.random_field((2, 3, g.nz, g.ny, g.nx), 19)
    ref = RC.fields(m, 2.0, U, G, 0.0) - RC.fields(m, 2.0, np.zeros_like(U), G, 0.0)
    f1, f0 = _fields(ctx, U, len(sites))
    got = f1 - f0
    for k in range(4):
        err = np.abs(got[..., k] - ref[..., k]).max() / np.abs(ref[..., k]).max()
        assert err <= 2e-6, (k, err)
    ctx.close()


def test_site_adjoint_is_the_transpose():
    """sum_r,k c[r,k] (F - F0)[r,k] = sum over cells of adjoint(c) . U for random c, U."""
    need_gpu()
    m = _model((6, 5, 2), seed=7)
    g = m.grid
    ctx = _ctx(m)
    sites = [(33.0, 20.0), (140.0, 201.0), (299.0, 80.0)]
    ctx.set_receivers_xy([s[0] for s in sites], [s[1] for s in sites], 0.0)
    U = W.random_field((2, 3, g.nz, g.ny, g.nx), 23)
    f1, f0 = _fields(ctx, U, len(sites))
    rng = np.random.default_rng(29)
    c = rng.standard_normal((2, len(sites), 4)) + 1j * rng.standard_normal((2, len(sites), 4))
    cd = to_dev(c)
    rhs = torch.empty((2, 3, g.nz, g.ny, g.nx), dtype=torch.complex128, device="cuda")
    ctx.receiver_adjoint(0, cd.data_ptr(), 2, rhs.data_ptr())
    lhs = np.sum(c * (f1 - f0), axis=(1, 2))
    rh = np.sum(to_host(rhs) * U, axis=(1, 2, 3, 4))
    assert np.max(np.abs(lhs - rh)) <= 1e-10 * np.max(np.abs(lhs))
    ctx.close()


def test_apparent_resistivity_and_phase():
    need_gpu()
    m = _model((4, 4, 2))
    ctx = _ctx(m)
    rng = np.random.default_rng(31)
    Z = (rng.standard_normal((9, 2, 2)) + 1j * rng.standard_normal((9, 2, 2))) * 1e-3
    zd = to_dev(Z)
    rho = torch.empty((9, 4), dtype=torch.float64, device="cuda")
    ph = torch.empty_like(rho)
    ctx.mt_apparent(0, zd.data_ptr(), 9, rho.data_ptr(), ph.data_ptr())
    r_ref, p_ref = RC.apparent(Z, 2.0)
    assert np.allclose(to_host(rho), r_ref.reshape(9, 4), rtol=1e-13, atol=0)
    assert np.allclose(to_host(ph), p_ref.reshape(9, 4), rtol=1e-13, atol=1e-12)
    ctx.close()


def test_site_outside_the_grid_is_rejected():
    need_gpu()
    from paper_1512_06126_gb300 import ie
    m = _model((4, 4, 2))
    ctx = _ctx(m)
    with pytest.raises(ie.IEError):
        ctx.set_receivers_xy([10.0, 201.0], [10.0, 10.0], 0.0)  # the grid spans x in [0, 200]
    ctx.close()
