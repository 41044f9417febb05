"""GPU receiver fields, MT misfit and its adjoint gradient against the oracle
(oracle/receivers.py), and the autograd Function against finite differences of the
GPU misfit itself."""
import numpy as np
import pytest

import workloads as W
from oracle import coefficients, receivers as RC
from tests.gpu_support import need_gpu, to_dev, to_host, torch
from tests.test_oracle_receivers import _tiny_problem

pytestmark = pytest.mark.gpu


def _ctx(model, problems=None, max_rhs=2):
    from paper_1512_06126_gb300 import build, ie
    build.build()
    g = model.grid
    q = None
    if problems is not None:
        q = [qa[g.ny - 1:, g.nx - 1:] for (_, qa, _, _) in problems]
    return ie.Context(g, model.layers, model.sigma_a, model.freqs, q, max_rhs=max_rhs)


@pytest.mark.parametrize("shape,rec", [((3, 3, 2), [(0, 0), (1, 1), (2, 1), (0, 2)]),
                                       ((7, 5, 3), [(0, 0), (6, 4), (3, 2), (1, 4), (5, 0)])])
def test_receiver_fields_against_oracle(shape, rec):
    """Scattered fields at the receivers (fields minus the fields of U = 0) for random
    U and a model with anomalies in every z-layer, against the oracle's dense
    receiver operator."""
    need_gpu()
    nx, ny, nz = shape
    layers = W.Layers((0.0, 140.0), (1e-9, 0.02, 0.005))
    grid = W.uniform_grid(nx, ny, nz, 50.0, z0=40.0)
    sb = W.background_sigma(grid, layers)
    rng = np.random.default_rng(3)
    sa = np.broadcast_to(sb[:, None, None], (nz, ny, nx)).astype(np.complex128).copy()
    mask = rng.random((nz, ny, nx)) < 0.6
    sa[mask] = 10 ** rng.uniform(-2, 0, mask.sum())
    m = W.Model("rx_f", grid, layers, sa, (2.0,), ("x", "y"))
    ctx = _ctx(m)
    iy = [r[1] for r in rec]
    ix = [r[0] for r in rec]
    ctx.set_receivers(ix, iy, 0.0)
    G = RC.receiver_operator(grid, layers, 2.0, 0.0, [(r[1], r[0]) for r in rec])
    U = W.random_field((2, 3, nz, ny, nx), 17)
    ref = RC.fields(m, 2.0, U, G, 0.0) - RC.fields(m, 2.0, np.zeros_like(U), G, 0.0)
    ud = to_dev(U)
    f1 = torch.empty((2, len(rec), 4), dtype=torch.complex128, device="cuda")
    f0 = torch.empty_like(f1)
    ctx.receiver_fields(0, ud.data_ptr(), 2, (0, 1), f1.data_ptr())
    ctx.receiver_fields(0, torch.zeros_like(ud).data_ptr(), 2, (0, 1), f0.data_ptr())
    got = to_host(f1) - to_host(f0)
    for k in range(4):
        err = np.abs(got[..., k] - ref[..., k]).max() / np.abs(ref[..., k]).max()
        assert err <= 2e-6, (shape, k, err)
    # the normal field alone: E_x (x-pol) and E_y (y-pol) equal the 1-D value
    En, Hn = RC.normal_at(layers, 2.0, 0.0)
    n0 = to_host(f0)
    assert np.allclose(n0[0, :, 0], En, rtol=1e-12) and np.allclose(n0[0, :, 3], Hn, rtol=1e-12)
    assert np.allclose(n0[1, :, 1], En, rtol=1e-12) and np.allclose(n0[1, :, 2], -Hn, rtol=1e-12)
    ctx.close()


def test_misfit_and_gradient_against_oracle():
    """Phi and dPhi/dln(sigma_a) of the whole pipeline (FP64 solves) against the
    oracle's dense-LU values on the tiny two-frequency problem."""
    need_gpu()
    from paper_1512_06126_gb300 import ie, mt
    m, problems, zobs = _tiny_problem()
    phi_ref = RC.misfit_of(m, problems, zobs)
    g_ref = RC.gradient(m, problems, zobs)
    ctx = _ctx(m, problems)
    rec = [(0, 0), (1, 1), (2, 1), (0, 2)]        # (iy, ix) as in the oracle problem
    P = mt.MTProblem(ctx, [r[1] for r in rec], [r[0] for r in rec], np.stack(zobs), tol=1e-12)
    phi = P.misfit()
    g = P.gradient().cpu().numpy()
    assert abs(phi - phi_ref) <= 1e-6 * phi_ref, (phi, phi_ref)
    an = g_ref != 0
    assert np.all(g[~an] == 0.0)
    err = np.abs(g[an] - g_ref[an]).max() / np.abs(g_ref[an]).max()
    assert err <= 1e-5, (err, g[an], g_ref[an])
    ctx.close()


@pytest.mark.parametrize("store", [True, False])
def test_autograd_function_matches_finite_differences(store):
    """torch.autograd through MTMisfit: backward equals a central difference of the GPU
    misfit along a random direction (h = 1e-4 in ln sigma); with store=False the
    forward fields are recomputed in backward."""
    need_gpu()
    from paper_1512_06126_gb300 import mt
    m, problems, zobs = _tiny_problem()
    ctx = _ctx(m, problems)
    rec = [(0, 0), (1, 1), (2, 1), (0, 2)]
    P = mt.MTProblem(ctx, [r[1] for r in rec], [r[0] for r in rec], np.stack(zobs), tol=1e-12, store_fields=store)
    sb = W.background_sigma(m.grid, m.layers)
    base = np.broadcast_to(sb[:, None, None], m.sigma_a.shape).astype(np.complex128).copy()
    cells = np.flatnonzero(np.abs(m.sigma_a - base).reshape(-1) > 0)
    theta = torch.tensor(np.log(m.sigma_a.reshape(-1)[cells].real), dtype=torch.float64, requires_grad=True)
    phi = mt.MTMisfit.apply(theta, P, cells, base)
    phi.backward()
    d = torch.tensor(np.random.default_rng(2).standard_normal(len(cells)), dtype=torch.float64)
    h = 1e-4
    with torch.no_grad():
        pp = mt.MTMisfit.apply(theta + h * d, P, cells, base)
        pm = mt.MTMisfit.apply(theta - h * d, P, cells, base)
    fd = float((pp - pm) / (2 * h))
    an = float(theta.grad @ d)
    assert abs(an - fd) <= 1e-5 * abs(fd), (an, fd)
    ctx.close()
