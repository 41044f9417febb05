"""Batched solves over several frequencies of one grid, the contraction variants and
their autotuner, through the C ABI."""
import numpy as np
import pytest

import workloads as W
from oracle import normal, operator as O
from tests.gpu_support import need_gpu, rel, to_dev, to_host, torch
from tests.oracle_cache import all_offsets_cached

pytestmark = pytest.mark.gpu


def _lib():
    from paper_1512_06126_gb300 import build, ie
    build.build()
    return ie


@pytest.mark.parametrize("precision,tol,bound", [(0, 1e-10, 1e-9), (1, 1e-7, 1e-5), (2, 1e-7, 1e-5)])
@pytest.mark.parametrize("adjoint", [False, True])
def test_batch_solve_against_lu(precision, tol, bound, adjoint):
    """Three frequencies x two polarisations in one lockstep solve; every block
    against a dense LU solve of its own operator (A or A^T)."""
    need_gpu()
    ie = _lib()
    base = W.small_model(nx=7, ny=5, nz=3, seed=11, freq=3.0)
    freqs = (0.3, 3.0, 30.0)
    qs, As, bs = [], [], []
    for f in freqs:
        m = W.Model(base.name, base.grid, base.layers, base.sigma_a, (f,), ("x", "y"))
        qa = all_offsets_cached(m)
        qs.append(qa[m.grid.ny - 1:, m.grid.nx - 1:])
        A = O.dense_matrix(m, O.dense_B(m, qa))
        As.append(A.T if adjoint else A)
        bs.append(np.stack([normal.rhs_U0(m, f, "x"), normal.rhs_U0(m, f, "y")]))
    g = base.grid
    ctx = ie.Context(g, base.layers, base.sigma_a, freqs, qs, max_rhs=6)
    b = np.stack(bs)                                   # [3][2][3][Nz][Ny][Nx]
    bd = to_dev(b)
    ud = torch.zeros_like(bd)
    torch.cuda.synchronize()
    st, info = ctx.solve_batch([0, 1, 2], bd.data_ptr(), ud.data_ptr(), 2, tol, precision=precision, adjoint=adjoint)
    assert st == 0, (st, info.final_rel_res)
    u = to_host(ud)
    for k in range(3):
        for p in range(2):
            ref = np.linalg.solve(As[k], b[k, p].ravel()).reshape(b[k, p].shape)
            assert rel(u[k, p], ref) <= bound, (k, p, rel(u[k, p], ref))
    # the same instances solved one at a time agree with the batch
    for k in (0, 2):
        u1 = torch.zeros_like(bd[k])
        st, _ = ctx.solve(k, bd[k].data_ptr(), u1.data_ptr(), 2, tol, precision=precision, adjoint=adjoint)
        assert st == 0
        assert rel(to_host(u1), u[k]) <= 10 * bound
    ctx.close()


@pytest.mark.parametrize("shape", [(24, 20, 32), (20, 16, 24), (12, 10, 48)])
def test_contract_variants_agree(shape):
    """Every applicable c64 contraction variant (forced) against the c128 product on
    generated coefficients, and bit-identical on repeat; the autotuner's choice is
    one of them and was timed."""
    need_gpu()
    ie = _lib()
    nx, ny, nz = shape
    m = W.small_model(nx=nx, ny=ny, nz=nz, seed=3, freq=1.0)
    g = m.grid
    ctx = ie.Context(g, m.layers, m.sigma_a, m.freqs[:1], None, max_rhs=2)
    variants, ms = ctx.contract_tuning()
    s = torch.cuda.current_stream().cuda_stream
    for R in (1, 2):
        assert 0 <= variants[R - 1] < ie.N_CONTRACT_VARIANTS
        assert ms[R - 1, variants[R - 1]] > 0 or ms[R - 1].max() == 0
        x = W.random_field((R, 3, nz, ny, nx), 50 + R)
        x128 = to_dev(x.astype(np.complex64).astype(np.complex128))
        y128 = torch.empty_like(x128)
        ctx.matvec(0, x128.data_ptr(), y128.data_ptr(), R, dtype=1, stream=s)
        x64 = x128.to(torch.complex64)
        tried = 0
        for v in range(ie.N_CONTRACT_VARIANTS):
            try:
                ctx.set_contract_variant(R, v)
            except ie.IEError:
                continue
            tried += 1
            y1 = torch.empty_like(x64)
            y2 = torch.empty_like(x64)
            ctx.matvec(0, x64.data_ptr(), y1.data_ptr(), R, dtype=0, stream=s)
            ctx.matvec(0, x64.data_ptr(), y2.data_ptr(), R, dtype=0, stream=s)
            torch.cuda.synchronize()
            assert torch.equal(y1, y2), (shape, R, v)
            err = float((y1.to(torch.complex128) - y128).norm() / y128.norm())
            assert err <= 2e-6, (shape, R, v, err)
        assert tried >= 2
    ctx.close()
