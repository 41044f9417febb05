"""GPU checks of the entry points around the product: the in-cell field E = U / a
(ie_fields) against the oracle, and the error path of the contraction's bounded
waits (IE_ERR_TIMEOUT reported by ie_sync and by the solves, the context usable
afterwards).  The waits are made to run out through the testing aid
ie_debug_set_wait_limit(0): every main wait then gives up at once, each kernel
drains its own copies in flight with the default limit and returns, so no GPU
fault or hang is involved."""
import numpy as np
import pytest

import workloads as W
from oracle import normal, operator as O
from tests.gpu_support import lib_context, need_gpu, rel, to_dev, to_host, torch
from tests.oracle_cache import all_offsets_cached

pytestmark = pytest.mark.gpu


def test_fields_against_oracle():
    need_gpu()
    m = W.small_model(nx=7, ny=5, nz=3, seed=11, freq=3.0)
    g = m.grid
    q = all_offsets_cached(m)[g.ny - 1:, g.nx - 1:]
    ctx = lib_context(m, [q], max_rhs=2)
    U = W.random_field((2, 3, g.nz, g.ny, g.nx), 17)
    ud = to_dev(U)
    ed = torch.empty_like(ud)
    ctx.fields(ud.data_ptr(), ed.data_ptr(), 2)
    assert rel(to_host(ed), O.in_cell_field(m, U)) <= 1e-14
    # in place, on a solved field: E of the solution of the x-polarised plane wave
    b = to_dev(normal.rhs_U0(m, m.freqs[0], "x")[None])
    u = torch.zeros_like(b)
    st, info = ctx.solve(0, b.data_ptr(), u.data_ptr(), 1, 1e-10, precision=0)
    assert st == 0
    uh = to_host(u)
    ctx.fields(u.data_ptr(), u.data_ptr(), 1)
    assert rel(to_host(u), O.in_cell_field(m, uh)) <= 1e-14
    ctx.close()


def _ctx_nz16():
    m = W.small_model(nx=20, ny=16, nz=16, seed=3, freq=1.0)
    g = m.grid
    q = W.random_compressed_q(g.ny, g.nx, g.nz, seed=31)
    return m, q, lib_context(m, [q], max_rhs=2)


@pytest.mark.parametrize("variant", [0, 1, 3, 4, 5, 6, 7])
def test_timed_out_contraction_is_reported_by_sync(variant):
    need_gpu()
    from paper_1512_06126_gb300 import ie
    m, q, ctx = _ctx_nz16()
    g = m.grid
    R = 2
    ctx.set_contract_variant(R, variant)
    x = W.random_field((R, 3, g.nz, g.ny, g.nx), 5)
    xd = to_dev(x, torch.complex64)
    yd = torch.empty_like(xd)
    try:
        ie.debug_set_wait_limit(0)
        ctx.matvec(0, xd.data_ptr(), yd.data_ptr(), R, dtype=ie.IE_C64)
        assert ctx.sync() == ie.IE_ERR_TIMEOUT
    finally:
        ie.debug_set_wait_limit(-1)
    # the word is cleared and the context still works
    assert ctx.sync() == ie.IE_OK
    ctx.matvec(0, xd.data_ptr(), yd.data_ptr(), R, dtype=ie.IE_C64)
    assert ctx.sync() == ie.IE_OK
    qt = O.full_spectrum_blocks(O.embed_spectrum(q))
    y = to_host(yd).astype(np.complex128)
    for r in range(R):
        ref = O.fft_apply(m, qt, x[r].astype(np.complex64).astype(np.complex128))
        assert rel(y[r], ref) <= 2e-5
    ctx.close()


@pytest.mark.parametrize("precision", [1, 2])
def test_timed_out_contraction_fails_the_solve(precision):
    need_gpu()
    from paper_1512_06126_gb300 import ie
    m, q, ctx = _ctx_nz16()
    g = m.grid
    ctx.set_contract_variant(2, 5)
    b = to_dev(W.random_field((2, 3, g.nz, g.ny, g.nx), 8))
    u = torch.zeros_like(b)
    try:
        ie.debug_set_wait_limit(0)
        with pytest.raises(ie.IEError) as e:
            ctx.solve(0, b.data_ptr(), u.data_ptr(), 2, 1e-7, precision=precision)
        assert e.value.status == ie.IE_ERR_TIMEOUT
    finally:
        ie.debug_set_wait_limit(-1)
    u.zero_()
    st, info = ctx.solve(0, b.data_ptr(), u.data_ptr(), 2, 1e-7, precision=precision)
    assert st == 0 and info.final_rel_res <= 1e-7
    ctx.close()
