"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (relative L2 unless stated):
* c128 matrix-vector product: 1e-12 (FFT round-off of two routes, O(eps log N)).
* c64 product: 2e-5 (FP32 FFTs and contraction with FP32 accumulation: about
  eps32 * (log2(4 Nx Ny) + 3 Nz) for these sizes, where eps32 = 6e-8).
* FP64 solve at tol 1e-10: 1e-9 against dense LU (cond(A) of the small models <~ 10).
* mixed solve at tol 1e-7: 1e-5 on U against dense LU.
"""
import numpy as np
import pytest

import workloads as W
from oracle import normal, operator as O
from tests.gpu_support import lib_context, need_gpu, rel, to_dev, to_host, torch
from tests.oracle_cache import all_offsets_cached

pytestmark = pytest.mark.gpu

MODELS = {
    "c1": lambda: W.config1(),
    "ragged": lambda: W.small_model(nx=7, ny=5, nz=3, seed=11, freq=3.0),
    "nz1": lambda: W.small_model(nx=6, ny=6, nz=1, seed=5, freq=0.5, n_layers=1),
}


@pytest.fixture(scope="module", params=list(MODELS))
def case(request):
    need_gpu()
    m = MODELS[request.param]()
    qa = all_offsets_cached(m)
    g = m.grid
    q = qa[g.ny - 1:, g.nx - 1:]
    B = O.dense_B(m, qa)
    A = O.dense_matrix(m, B)
    ctx = lib_context(m, [q], max_rhs=2)
    yield m, q, A, ctx
    ctx.close()


def test_matvec_c128_and_transpose(case):
    m, q, A, ctx = case
    g = m.grid
    shp = (2, 3, g.nz, g.ny, g.nx)
    x = W.random_field(shp, 3)
    xd = to_dev(x)
    yd = torch.empty_like(xd)
    for tr in (False, True):
        ctx.matvec(0, xd.data_ptr(), yd.data_ptr(), 2, dtype=1, transpose=tr,
                   stream=torch.cuda.current_stream().cuda_stream)
        y = to_host(yd)
        M = A.T if tr else A
        for r in range(2):
            ref = (M @ x[r].ravel()).reshape(x[r].shape)
            assert rel(y[r], ref) <= 1e-12, (tr, r, rel(y[r], ref))


def test_matvec_c64(case):
    m, q, A, ctx = case
    g = m.grid
    x = W.random_field((1, 3, g.nz, g.ny, g.nx), 4)
    xd = to_dev(x, torch.complex64)
    yd = torch.empty_like(xd)
    ctx.matvec(0, xd.data_ptr(), yd.data_ptr(), 1, dtype=0, stream=torch.cuda.current_stream().cuda_stream)
    y = to_host(yd).astype(np.complex128)
    ref = (A @ x[0].astype(np.complex64).astype(np.complex128).ravel()).reshape(x[0].shape)
    assert rel(y[0], ref) <= 2e-5


def test_rhs_mt_matches_oracle(case):
    m, q, A, ctx = case
    for pol, name in ((0, "x"), (1, "y")):
        u0 = torch.empty((3, m.grid.nz, m.grid.ny, m.grid.nx), dtype=torch.complex128, device="cuda")
        ctx.rhs_mt(0, pol, u0.data_ptr())
        ref = normal.rhs_U0(m, m.freqs[0], name)
        assert rel(to_host(u0), ref) <= 1e-12


@pytest.mark.parametrize("precision,tol,bound", [(0, 1e-10, 1e-9), (1, 1e-7, 1e-5), (2, 1e-7, 1e-5)])
def test_solve_against_lu(case, precision, tol, bound):
    m, q, A, ctx = case
    g = m.grid
    b = np.stack([normal.rhs_U0(m, m.freqs[0], "x"), normal.rhs_U0(m, m.freqs[0], "y")])
    u_ref = np.stack([np.linalg.solve(A, b[r].ravel()).reshape(b[r].shape) for r in range(2)])
    bd = to_dev(b)
    ud = torch.zeros_like(bd)
    torch.cuda.synchronize()
    st, info = ctx.solve(0, bd.data_ptr(), ud.data_ptr(), 2, tol, precision=precision)
    assert st == 0, (st, info.final_rel_res)
    assert info.final_rel_res <= tol
    u = to_host(ud)
    for r in range(2):
        assert rel(u[r], u_ref[r]) <= bound, (r, rel(u[r], u_ref[r]))


def test_adjoint_solve_against_lu(case):
    m, q, A, ctx = case
    g = m.grid
    b = W.random_field((1, 3, g.nz, g.ny, g.nx), 9)
    w_ref = np.linalg.solve(A.T, b[0].ravel()).reshape(b[0].shape)
    bd = to_dev(b)
    wd = torch.zeros_like(bd)
    torch.cuda.synchronize()
    st, info = ctx.solve(0, bd.data_ptr(), wd.data_ptr(), 1, 1e-10, precision=0, adjoint=True)
    assert st == 0
    assert rel(to_host(wd)[0], w_ref) <= 1e-9


def test_no_anomaly_solution_is_normal_field():
    need_gpu()
    m0 = W.small_model(nx=5, ny=4, nz=3, seed=11, freq=3.0)
    sb = W.background_sigma(m0.grid, m0.layers)
    m = W.Model(m0.name, m0.grid, m0.layers, np.broadcast_to(sb[:, None, None], m0.sigma_a.shape).copy(),
                m0.freqs, m0.pols)
    qa = all_offsets_cached(m0)
    q = qa[m.grid.ny - 1:, m.grid.nx - 1:]
    ctx = lib_context(m, [q], max_rhs=1)
    b = normal.rhs_U0(m, m.freqs[0], "x")[None]
    bd = to_dev(b)
    ud = torch.zeros_like(bd)
    torch.cuda.synchronize()
    st, info = ctx.solve(0, bd.data_ptr(), ud.data_ptr(), 1, 1e-12, precision=0)
    # A = I when gamma = 0: one Krylov step from the zero guess reaches U = U^0
    assert st == 0 and info.inner_iters == 1
    assert rel(to_host(ud), b) <= 1e-15
    # starting from U^0 itself no iteration is needed
    ud2 = bd.clone()
    st, info = ctx.solve(0, bd.data_ptr(), ud2.data_ptr(), 1, 1e-12, precision=0, use_x0=True)
    assert st == 0 and info.inner_iters == 0
    assert rel(to_host(ud2), b) == 0.0
    ctx.close()


def test_full_size_matvec_sampled_rows():
    """128 x 128 x 32 (the single-solve grid) with a random coefficient tensor:
    sampled rows of A x from direct summation in the oracle."""
    need_gpu()
    m = W.config2()
    g = m.grid
    q = W.random_compressed_q(g.ny, g.nx, g.nz, seed=21)
    ctx = lib_context(m, [q], max_rhs=2)
    x = W.random_field((2, 3, g.nz, g.ny, g.nx), 22)
    xd = to_dev(x)
    yd = torch.empty_like(xd)
    ctx.matvec(0, xd.data_ptr(), yd.data_ptr(), 2, dtype=1, stream=torch.cuda.current_stream().cuda_stream)
    y = to_host(yd)
    x32 = to_dev(x, torch.complex64)
    y32 = torch.empty_like(x32)
    ctx.matvec(0, x32.data_ptr(), y32.data_ptr(), 2, dtype=0, stream=torch.cuda.current_stream().cuda_stream)
    y32h = to_host(y32).astype(np.complex128)
    cells = [(0, 0, 0), (31, 127, 127), (5, 64, 3), (17, 1, 126), (31, 0, 77)]
    for r in range(2):
        ref = O.direct_rows(m, q, x[r], cells)
        got = np.array([y[r][:, c[0], c[1], c[2]] for c in cells])
        assert rel(got, ref) <= 1e-11, rel(got, ref)
        got32 = np.array([y32h[r][:, c[0], c[1], c[2]] for c in cells])
        # the c64 bound of every other product test, on 15 sampled values: the FFT
        # round-off spreads evenly over the output, so sampled rows of typical size see
        # the same relative error as the whole vector
        assert rel(got32, ref) <= 2e-5, rel(got32, ref)
    ctx.close()


@pytest.mark.parametrize("shape", [(40, 24, 16), (20, 36, 24), (16, 12, 48), (24, 20, 32)])
def test_c64_pipelined_contraction_against_c128(shape):
    """The pipelined c64 contraction (Nz in {16, 24, 32, 48}) against the c128 path and
    the oracle's FFT apply, on a random coefficient tensor with the physical layout."""
    need_gpu()
    nx, ny, nz = shape
    m0 = W.small_model(nx=nx, ny=ny, nz=nz, seed=3, freq=1.0)
    g = m0.grid
    q = W.random_compressed_q(ny, nx, nz, seed=31)
    ctx = lib_context(m0, [q], max_rhs=2)
    qt = O.full_spectrum_blocks(O.embed_spectrum(q))
    for R in (1, 2):
        x = W.random_field((R, 3, nz, ny, nx), 32 + R)
        xd = to_dev(x, torch.complex64)
        yd = torch.empty_like(xd)
        ctx.matvec(0, xd.data_ptr(), yd.data_ptr(), R, dtype=0, stream=torch.cuda.current_stream().cuda_stream)
        y = to_host(yd).astype(np.complex128)
        for r in range(R):
            ref = O.fft_apply(m0, qt, x[r].astype(np.complex64).astype(np.complex128))
            assert rel(y[r], ref) <= 2e-5, (shape, R, r, rel(y[r], ref))
    ctx.close()


@pytest.mark.parametrize("shape", [(24, 20, 32), (20, 16, 24), (12, 10, 48)])
def test_c128_double_float_contraction_matches_fp64(shape):
    """The c128 product with its contraction in compensated double-float arithmetic
    (the mixed solver's residuals) against the FP64 product on generated coefficients,
    for 1, 2 and 4 right-hand sides and both transposes.  Bound: the compensated dot
    product is as accurate as one in twice FP32 precision, an error of about
    (3 Nz eps32)^2 ~ 3e-11 of the sum of magnitudes at Nz = 32; 1e-10 relative to the
    whole product leaves a margin for the FFTs' own FP64 error (~1e-15)."""
    need_gpu()
    nx, ny, nz = shape
    m0 = W.small_model(nx=nx, ny=ny, nz=nz, seed=5, freq=1.0)
    g = m0.grid
    from paper_1512_06126_gb300 import build, ie
    build.build()
    ctx = ie.Context(g, m0.layers, m0.sigma_a, m0.freqs[:1], None, max_rhs=4)
    s = torch.cuda.current_stream().cuda_stream
    for R in (1, 2, 4):
        x = to_dev(W.random_field((R, 3, nz, ny, nx), 90 + R), torch.complex128)
        for tr in (0, 1):
            y64 = torch.empty_like(x)
            ydf = torch.empty_like(x)
            ctx.matvec(0, x.data_ptr(), y64.data_ptr(), R, dtype=ie.IE_C128, transpose=tr, stream=s)
            ctx.matvec(0, x.data_ptr(), ydf.data_ptr(), R, dtype=ie.IE_C128_DF, transpose=tr, stream=s)
            torch.cuda.synchronize()
            err = float((ydf - y64).norm() / y64.norm())
            assert err <= 1e-10, (shape, R, tr, err)
    ctx.close()


@pytest.mark.parametrize("shape", [(24, 20, 32), (24, 20, 16), (20, 16, 24), (12, 10, 48)])
def test_c64_pipelined_contraction_generated_coefficients(shape):
    """The pipelined c64 contraction on coefficients from the device generator (the
    physical tensor, with its large self terms) against the c128 path, and two calls
    in a row bit-identical: a wrong or racy store in one row of one wavenumber shows
    here even where it hides under random coefficients.  FP32 bound: the contraction
    sums 3 Nz products and each FFT pass adds O(eps32 log N); 2e-6 leaves a margin of
    ~40x over the measured ~4e-8."""
    need_gpu()
    nx, ny, nz = shape
    m0 = W.small_model(nx=nx, ny=ny, nz=nz, seed=3, freq=1.0)
    g = m0.grid
    from paper_1512_06126_gb300 import build, ie
    build.build()
    ctx = ie.Context(g, m0.layers, m0.sigma_a, m0.freqs[:1], None, max_rhs=2)
    s = torch.cuda.current_stream().cuda_stream
    for R in (1, 2):
        x = W.random_field((R, 3, nz, ny, nx), 40 + R)
        x128 = to_dev(x.astype(np.complex64).astype(np.complex128), torch.complex128)
        y128 = torch.empty_like(x128)
        ctx.matvec(0, x128.data_ptr(), y128.data_ptr(), R, dtype=1, stream=s)
        x64 = x128.to(torch.complex64)
        y1 = torch.empty_like(x64)
        y2 = torch.empty_like(x64)
        ctx.matvec(0, x64.data_ptr(), y1.data_ptr(), R, dtype=0, stream=s)
        ctx.matvec(0, x64.data_ptr(), y2.data_ptr(), R, dtype=0, stream=s)
        torch.cuda.synchronize()
        assert torch.equal(y1, y2), (shape, R, float((y1 - y2).abs().max()))
        err = float((y1.to(torch.complex128) - y128).norm() / y128.norm())
        assert err <= 2e-6, (shape, R, err)
    ctx.close()


@pytest.mark.parametrize("shape", [(12, 10, 48), (8, 6, 64)])
def test_large_nz_contraction_against_oracle(shape):
    """Nz whose full 3 Nz x 3 Nz c128 block does not fit in shared memory: the
    panel-staged contraction (c128 always; c64 for R > 2 or Nz outside the pipelined
    set) against the oracle's FFT apply, R = 1..3."""
    need_gpu()
    nx, ny, nz = shape
    m0 = W.small_model(nx=nx, ny=ny, nz=nz, seed=5, freq=1.0)
    q = W.random_compressed_q(ny, nx, nz, seed=33)
    ctx = lib_context(m0, [q], max_rhs=3)
    qt = O.full_spectrum_blocks(O.embed_spectrum(q))
    x = W.random_field((3, 3, nz, ny, nx), 61)
    for R in (1, 2, 3):
        xd = to_dev(x[:R])
        yd = torch.empty_like(xd)
        ctx.matvec(0, xd.data_ptr(), yd.data_ptr(), R, dtype=1, stream=torch.cuda.current_stream().cuda_stream)
        y = to_host(yd)
        x32 = to_dev(x[:R], torch.complex64)
        y32d = torch.empty_like(x32)
        ctx.matvec(0, x32.data_ptr(), y32d.data_ptr(), R, dtype=0, stream=torch.cuda.current_stream().cuda_stream)
        y32 = to_host(y32d).astype(np.complex128)
        for r in range(R):
            ref = O.fft_apply(m0, qt, x[r])
            assert rel(y[r], ref) <= 1e-12, (shape, R, r, rel(y[r], ref))
            ref32 = O.fft_apply(m0, qt, x[r].astype(np.complex64).astype(np.complex128))
            assert rel(y32[r], ref32) <= 2e-5, (shape, R, r, rel(y32[r], ref32))
    ctx.close()


@pytest.mark.parametrize("precision,tol,bound", [(0, 1e-10, 1e-9), (1, 1e-7, 1e-6), (2, 1e-7, 1e-6)])
def test_solve_weak_contrast_takes_second_projection(precision, tol, bound):
    """A weak anomaly (sigma_a = sigma_b (1 + 1e-6)) makes A = I + O(1e-6): each new
    Krylov vector A v_k is v_k up to a part of relative size ~1e-6, so the first
    Gram-Schmidt projection cancels nearly all of it and the second projection runs.
    The solution must still match a dense LU solve."""
    need_gpu()
    m = W.small_model(nx=7, ny=5, nz=3, seed=11, freq=3.0)
    g = m.grid
    sb = W.background_sigma(g, m.layers)
    sa = np.broadcast_to(sb[:, None, None], (g.nz, g.ny, g.nx)).astype(np.complex128).copy()
    sa[:, 1:4, 2:6] *= 1.0 + 1e-6
    m = W.Model(m.name, g, m.layers, sa, m.freqs, m.pols)
    qa = all_offsets_cached(m)
    q = qa[g.ny - 1:, g.nx - 1:]
    A = O.dense_matrix(m, O.dense_B(m, qa))
    b = np.stack([W.random_field((3, g.nz, g.ny, g.nx), 71 + r) for r in range(2)])
    u_ref = np.stack([np.linalg.solve(A, b[r].ravel()).reshape(b[r].shape) for r in range(2)])
    ctx = lib_context(m, [q], max_rhs=2)
    bd = to_dev(b)
    ud = torch.zeros_like(bd)
    torch.cuda.synchronize()
    st, info = ctx.solve(0, bd.data_ptr(), ud.data_ptr(), 2, tol, precision=precision)
    assert st == 0, (st, info.final_rel_res)
    assert info.reorth > 0, info.reorth
    u = to_host(ud)
    for r in range(2):
        assert rel(u[r], u_ref[r]) <= bound, (r, rel(u[r], u_ref[r]))
    ctx.close()


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_solve_nan_rhs_is_not_converged(precision):
    """A right-hand side holding a NaN must not come back as a converged solve (a NaN
    residual compares false against every tolerance)."""
    need_gpu()
    m = W.small_model(nx=7, ny=5, nz=3, seed=11, freq=3.0)
    g = m.grid
    qa = all_offsets_cached(m)
    q = qa[g.ny - 1:, g.nx - 1:]
    ctx = lib_context(m, [q], max_rhs=2)
    b = np.stack([W.random_field((3, g.nz, g.ny, g.nx), 81 + r) for r in range(2)])
    b[1, 2, 1, 2, 3] = np.nan
    bd = to_dev(b)
    ud = torch.zeros_like(bd)
    torch.cuda.synchronize()
    st, info = ctx.solve(0, bd.data_ptr(), ud.data_ptr(), 2, 1e-7, precision=precision)
    assert st != 0, (st, info.final_rel_res)
    assert not info.final_rel_res <= 1e-7
    ctx.close()


@pytest.mark.parametrize("shape", [(64, 64, 6), (128, 64, 4), (256, 32, 3), (64, 128, 5), (96, 96, 3),
                                   (192, 96, 2), (96, 192, 2)])
def test_fast_fft_lengths_against_c128(shape):
    """Grids whose padded lengths 2N are 128, 192, 256, 384 or 512 take the
    register-blocked FP32 FFTs (192 and 384 with a radix-3 step); the c64 product (one
    and two right-hand sides) must match the oracle's FFT product (2e-5) and the c128
    product, which uses the generic Stockham FFTs in FP64 (2e-6).  The mixed-precision
    solve (inner GMRES in c64 through the same FFTs) must reach the FP64 solve's
    solution."""
    need_gpu()
    nx, ny, nz = shape
    m0 = W.small_model(nx=nx, ny=ny, nz=nz, seed=7, freq=1.0)
    g = m0.grid
    q = W.random_compressed_q(ny, nx, nz, seed=41, decay=0.02)
    qt = O.full_spectrum_blocks(O.embed_spectrum(q))
    ctx = lib_context(m0, [q], max_rhs=2)
    s = torch.cuda.current_stream().cuda_stream
    for R in (1, 2):
        x = W.random_field((R, 3, nz, ny, nx), 60 + R)
        xr = x.astype(np.complex64).astype(np.complex128)
        x128 = to_dev(xr)
        y128 = torch.empty_like(x128)
        ctx.matvec(0, x128.data_ptr(), y128.data_ptr(), R, dtype=1, stream=s)
        x64 = x128.to(torch.complex64)
        y64 = torch.empty_like(x64)
        ctx.matvec(0, x64.data_ptr(), y64.data_ptr(), R, dtype=0, stream=s)
        torch.cuda.synchronize()
        err = float((y64.to(torch.complex128) - y128).norm() / y128.norm())
        assert err <= 2e-6, (shape, R, err)
        y = to_host(y64).astype(np.complex128)
        for r in range(R):
            err = rel(y[r], O.fft_apply(m0, qt, xr[r]))
            assert err <= 2e-5, (shape, R, r, err)
    b = to_dev(np.stack([normal.rhs_U0(m0, 1.0, "x"), normal.rhs_U0(m0, 1.0, "y")]))
    u64 = torch.zeros_like(b)
    umx = torch.zeros_like(b)
    torch.cuda.synchronize()
    st, _ = ctx.solve(0, b.data_ptr(), u64.data_ptr(), 2, 1e-9, precision=0)
    assert st == 0
    st, _ = ctx.solve(0, b.data_ptr(), umx.data_ptr(), 2, 1e-7, precision=1)
    assert st == 0
    assert rel(to_host(umx), to_host(u64)) <= 1e-5
    ctx.close()


def test_fft_plans_against_oracle():
    """The plan autotuner's choice multiplies out to each transform length, and every
    stage order (radix 8, 4, 2, 3, 5 stages, odd factors first or last), set by hand,
    gives the oracle's FFT product: c128 at 1e-12, c64 (generic FP32 Stockham: 2Nx = 96
    and 2Ny = 80 have no register-blocked kernel) at 2e-5."""
    need_gpu()
    from paper_1512_06126_gb300 import ie
    nx, ny, nz = 48, 40, 2
    m = W.small_model(nx=nx, ny=ny, nz=nz, seed=5, freq=1.0)
    q = W.random_compressed_q(ny, nx, nz, seed=43, decay=0.02)
    qt = O.full_spectrum_blocks(O.embed_spectrum(q))
    ctx = lib_context(m, [q], max_rhs=1)
    for axis, L in ((0, 2 * nx), (1, 2 * ny)):
        r, ms = ctx.fft_plan(axis)
        assert int(np.prod(r)) == L and set(r) <= {2, 3, 4, 5, 8}, (axis, r)
        assert ms > 0
    with pytest.raises(ie.IEError):
        ctx.set_fft_plan(0, [16, 6])  # 16 is not a radix of the kernels
    with pytest.raises(ie.IEError):
        ctx.set_fft_plan(1, [4, 4, 4])  # 64 != 2 Ny
    x = W.random_field((1, 3, nz, ny, nx), 71).astype(np.complex64).astype(np.complex128)
    ref = O.fft_apply(m, qt, x[0])
    xd = to_dev(x)
    s = torch.cuda.current_stream().cuda_stream
    plans_x = [[4, 4, 2, 3], [8, 4, 3], [3, 8, 4], [2, 4, 4, 3], [3, 2, 2, 2, 2, 2]]
    plans_y = [[4, 4, 5], [8, 2, 5], [5, 4, 4], [5, 8, 2], [2, 8, 5]]
    for px, py in zip(plans_x, plans_y):
        ctx.set_fft_plan(0, px)
        ctx.set_fft_plan(1, py)
        assert ctx.fft_plan(0)[0] == px and ctx.fft_plan(1)[0] == py
        yd = torch.empty_like(xd)
        ctx.matvec(0, xd.data_ptr(), yd.data_ptr(), 1, dtype=ie.IE_C128, stream=s)
        assert rel(to_host(yd)[0], ref) <= 1e-12, (px, py)
        x64 = xd.to(torch.complex64)
        y64 = torch.empty_like(x64)
        ctx.matvec(0, x64.data_ptr(), y64.data_ptr(), 1, dtype=ie.IE_C64, stream=s)
        assert rel(to_host(y64)[0].astype(np.complex128), ref) <= 2e-5, (px, py)
    ctx.close()
