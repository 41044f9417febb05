"""The allocation-free product ie_matvec_noalloc against ie_matvec.

ie_matvec_noalloc serves callers that may not allocate device memory: it takes every
operand as a device pointer and keeps its FFT work arrays in a fixed device array
owned by the library.  Here its output is compared with the context-based
ie_matvec (c64) on the same operator, on two consecutive calls with different
inputs (the second call must not see the first call's leftovers), within the c64
tolerance of the other GPU tests (2e-5 relative).  This file is collected last so
that a run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

import workloads as W
from oracle import operator as O
from tests.gpu_support import lib_context, need_gpu, rel, to_dev, to_host, torch
from tests.oracle_cache import all_offsets_cached

pytestmark = pytest.mark.gpu


def folded_spectral_c64(q):
    """Pack the DFT of the 2N-periodic embedding of q into the folded layout of
    ie_matvec_noalloc: [(Ny+1)(Nx+1)][2Nz(2Nz+1)] complex64."""
    ny, nx, _, nz, _ = q.shape
    qt = O.embed_spectrum(q)                       # [2Ny][2Nx][6][Nz][Nz]
    iu = np.triu_indices(nz)
    out = []
    for ky in range(ny + 1):
        for kx in range(nx + 1):
            b = qt[ky, kx]
            out.append(np.concatenate([b[0][iu], b[1][iu], b[2][iu], b[3][iu], b[4].ravel(), b[5].ravel()]))
    return np.asarray(out, dtype=np.complex64)


def scales(model):
    g = model.grid
    gamma, s, V = O.diagonals(model)
    cell = gamma.shape
    in_s = (s[:, None, None] * gamma).astype(np.complex64)
    out_s = np.broadcast_to((-(2.0 * s / V) / (4.0 * g.nx * g.ny))[:, None, None], cell).astype(np.complex64)
    diag = (1.0 - gamma).astype(np.complex64)
    return in_s, out_s, diag


@pytest.mark.parametrize("case", ["ragged", "nz16"])
def test_noalloc_matches_matvec_on_two_calls(case):
    need_gpu()
    from paper_1512_06126_gb300 import ie
    if case == "ragged":
        m = W.small_model(nx=7, ny=5, nz=3, seed=11, freq=3.0)
        q = all_offsets_cached(m)[m.grid.ny - 1:, m.grid.nx - 1:]
    else:
        m = W.small_model(nx=24, ny=20, nz=16, seed=3, freq=1.0)
        q = W.random_compressed_q(20, 24, 16, seed=31)
    g = m.grid
    R = 2
    ctx = lib_context(m, [q], max_rhs=R)
    qf = to_dev(folded_spectral_c64(q), torch.complex64)
    in_s, out_s, diag = (to_dev(a, torch.complex64) for a in scales(m))
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        x = W.random_field((R, 3, g.nz, g.ny, g.nx), 100 + call)
        xd = to_dev(x, torch.complex64)
        y_ref = torch.empty_like(xd)
        y_new = torch.full_like(xd, complex(float("nan"), 0.0))
        torch.cuda.synchronize()
        ctx.matvec(0, xd.data_ptr(), y_ref.data_ptr(), R, dtype=ie.IE_C64)
        torch.cuda.synchronize()
        st = ie.matvec_noalloc(g.nx, g.ny, g.nz, R, qf.data_ptr(), in_s.data_ptr(), out_s.data_ptr(),
                               diag.data_ptr(), xd.data_ptr(), y_new.data_ptr(), stream)
        assert st == ie.IE_OK, ie.status_str(st)
        a, b = to_host(y_new).astype(np.complex128), to_host(y_ref).astype(np.complex128)
        assert np.all(np.isfinite(a))
        assert rel(a, b) <= 2e-5, (case, call, rel(a, b))
        # and against the oracle's FFT product of the same (c64-rounded) input
        qt = O.full_spectrum_blocks(O.embed_spectrum(q))
        for r in range(R):
            ref = O.fft_apply(m, qt, x[r].astype(np.complex64).astype(np.complex128))
            assert rel(a[r], ref) <= 2e-5, (case, call, r, rel(a[r], ref))
    assert ie.noalloc_sync(stream) == ie.IE_OK
    ctx.close()


def test_noalloc_rejects_problems_above_the_work_space():
    need_gpu()
    from paper_1512_06126_gb300 import build, ie
    build.build()
    # 256 x 256 x 64 with two right-hand sides needs ~2.4 GB of work space
    d = torch.zeros(16, dtype=torch.complex64, device="cuda")
    p = d.data_ptr()
    st = ie.matvec_noalloc(256, 256, 64, 2, p, p, p, p, p, p + 8, None)
    assert st == ie.IE_ERR_SCRATCH


def test_noalloc_rejects_shapes_the_contraction_cannot_stage():
    """Four right-hand sides over 300 layers fit the work space (a 1 x 1 grid) but not
    the contraction's shared-memory staging: an argument error before any launch."""
    need_gpu()
    from paper_1512_06126_gb300 import build, ie
    build.build()
    d = torch.zeros(16, dtype=torch.complex64, device="cuda")
    p = d.data_ptr()
    assert ie.matvec_noalloc(1, 1, 300, 4, p, p, p, p, p, p + 8, None) == ie.IE_ERR_ARG
    assert ie.noalloc_sync(None) == ie.IE_OK


def test_noalloc_reports_a_timed_out_contraction():
    """With every main wait of the contraction giving up at once (testing aid), the
    call still returns IE_OK (it is asynchronous) and ie_noalloc_sync reports
    IE_ERR_TIMEOUT once; a later call with the default limit is exact again."""
    need_gpu()
    from paper_1512_06126_gb300 import ie
    m = W.small_model(nx=24, ny=20, nz=16, seed=3, freq=1.0)
    q = W.random_compressed_q(20, 24, 16, seed=31)
    g = m.grid
    R = 2
    qf = to_dev(folded_spectral_c64(q), torch.complex64)
    in_s, out_s, diag = (to_dev(a, torch.complex64) for a in scales(m))
    x = W.random_field((R, 3, g.nz, g.ny, g.nx), 7)
    xd = to_dev(x, torch.complex64)
    yd = torch.empty_like(xd)
    stream = torch.cuda.current_stream().cuda_stream
    args = (g.nx, g.ny, g.nz, R, qf.data_ptr(), in_s.data_ptr(), out_s.data_ptr(), diag.data_ptr(),
            xd.data_ptr(), yd.data_ptr(), stream)
    try:
        ie.debug_set_wait_limit(0)
        assert ie.matvec_noalloc(*args) == ie.IE_OK
        assert ie.noalloc_sync(stream) == ie.IE_ERR_TIMEOUT
    finally:
        ie.debug_set_wait_limit(-1)
    assert ie.noalloc_sync(stream) == ie.IE_OK
    assert ie.matvec_noalloc(*args) == ie.IE_OK
    assert ie.noalloc_sync(stream) == ie.IE_OK
    qt = O.full_spectrum_blocks(O.embed_spectrum(q))
    y = to_host(yd).astype(np.complex128)
    for r in range(R):
        ref = O.fft_apply(m, qt, x[r].astype(np.complex64).astype(np.complex128))
        assert rel(y[r], ref) <= 2e-5

