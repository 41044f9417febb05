"""The library's device coefficient generator against the oracle's coefficients.

The two compute the same integrals (Appendices A-C) by different routes: the
oracle integrates every offset on its own lambda knots; the device generator
evaluates the vertical integrals once on a master grid uniform in ln(lambda) and
maps each offset's Gauss-Legendre knots onto it by 8-point Lagrange interpolation.
Tolerance: 1e-7 of the largest entry of each block kind (the interpolation error
is below 1e-10 for the smooth vertical integrals; the bound leaves room for the
different summation orders)."""
import numpy as np
import pytest

import workloads as W
from oracle import coefficients as C
from tests.gpu_support import lib_context, need_gpu, rel, to_host, torch
from tests.oracle_cache import all_offsets_cached

pytestmark = pytest.mark.gpu


def generated(model, freq):
    from paper_1512_06126_gb300 import build, ie
    build.build()
    g = model.grid
    q = torch.empty((g.ny, g.nx, 6, g.nz, g.nz), dtype=torch.complex128, device="cuda")
    torch.cuda.synchronize()
    ie.generate_coefficients(g, model.layers, freq, q.data_ptr())
    return to_host(q)


@pytest.mark.parametrize("name", ["c1", "ragged", "nz1"])
def test_generator_matches_oracle(name):
    need_gpu()
    m = {"c1": W.config1, "ragged": lambda: W.small_model(nx=7, ny=5, nz=3, seed=11, freq=3.0),
         "nz1": lambda: W.small_model(nx=6, ny=6, nz=1, seed=5, freq=0.5, n_layers=1)}[name]()
    g = m.grid
    qa = all_offsets_cached(m)
    q_ref = qa[g.ny - 1:, g.nx - 1:]
    q_gen = generated(m, m.freqs[0])
    for b in range(6):
        scale = np.abs(q_ref[:, :, b]).max()
        err = np.abs(q_gen[:, :, b] - q_ref[:, :, b]).max()
        assert err <= 1e-7 * scale, (name, b, err / scale)


def test_generator_full_size_sampled_offsets():
    """128 x 128 x 32 grid of the single-solve workload: sampled offsets."""
    need_gpu()
    m = W.config2()
    g = m.grid
    q_gen = generated(m, m.freqs[0])
    for (i, j) in [(0, 0), (1, 1), (0, 5), (17, 3), (127, 127)]:
        ref = C.offset_blocks(g, m.layers, m.freqs[0], i, j)
        for b in range(6):
            scale = np.abs(ref[b]).max()
            if scale == 0:
                continue
            err = np.abs(q_gen[i, j, b] - ref[b]).max()
            assert err <= 1e-7 * scale + 1e-12 * np.abs(ref[0]).max(), (i, j, b, err / scale)


def test_solve_with_generated_coefficients():
    need_gpu()
    m = W.config1()
    g = m.grid
    from oracle import normal, operator as O
    qa = all_offsets_cached(m)
    A = O.dense_matrix(m, O.dense_B(m, qa))
    b = normal.rhs_U0(m, m.freqs[0], "x")[None]
    u_ref = np.linalg.solve(A, b[0].ravel()).reshape(b[0].shape)
    from paper_1512_06126_gb300 import ie
    ctx = ie.Context(g, m.layers, m.sigma_a, m.freqs, None, max_rhs=1)
    bd = torch.from_numpy(b).to("cuda")
    ud = torch.zeros_like(bd)
    torch.cuda.synchronize()
    st, info = ctx.solve(0, bd.data_ptr(), ud.data_ptr(), 1, 1e-10, precision=0)
    ctx.close()
    assert st == 0
    assert rel(to_host(ud)[0], u_ref) <= 1e-6
