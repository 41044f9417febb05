"""ctypes binding of libie_gb300.so: the same entry points as include/ie.h.

Argument marshalling only: every step of the computation runs in the library's
CUDA kernels.  Device buffers are passed as raw pointers (for instance
``torch.Tensor.data_ptr()`` of a CUDA tensor); this module never falls back to a
CPU path and raises if the library cannot be loaded.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libie_gb300.so")

IE_OK, IE_NOT_CONVERGED, IE_BREAKDOWN = 0, 1, 2
IE_ERR_ARG = -1
IE_ERR_SCRATCH = -6
IE_ERR_TIMEOUT = -7
IE_C64, IE_C128 = 0, 1
N_CONTRACT_VARIANTS = 9
IE_C128_DF = 7
IE_FP64, IE_MIXED, IE_MIXED_FP64K = 0, 1, 2
IE_PROF_PRODUCT_C64, IE_PROF_PRODUCT_C128, IE_PROF_GS_C64, IE_PROF_GS_C128, IE_PROF_GIVENS = 2, 3, 4, 5, 6

EXPORTS = ("ie_setup", "ie_generate_coefficients", "ie_matvec_noalloc", "ie_noalloc_sync", "ie_matvec", "ie_sync",
           "ie_fields", "ie_debug_set_wait_limit", "ie_solve", "ie_adjoint_solve", "ie_solve_batch",
           "ie_contract_tuning", "ie_fft_plan", "ie_set_fft_plan", "ie_set_contract_variant", "ie_rhs_mt",
           "ie_set_sigma", "ie_set_receivers", "ie_set_receivers_xy", "ie_mt_apparent",
           "ie_receiver_fields", "ie_mt_misfit", "ie_receiver_adjoint", "ie_gradient_accumulate", "ie_ctx_stream",
           "ie_ctx_device_bytes", "ie_profile", "ie_profile_read", "ie_profile_matvec", "ie_kernel_launches",
           "ie_destroy", "ie_status_str")


class ie_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("hx", ctypes.c_double), ("hy", ctypes.c_double),
                ("z_edges_host", ctypes.POINTER(ctypes.c_double)),
                ("x0", ctypes.c_double), ("y0", ctypes.c_double)]


class ie_layers(ctypes.Structure):
    _fields_ = [("n_interfaces", ctypes.c_int),
                ("interfaces_host", ctypes.POINTER(ctypes.c_double)),
                ("sigma_host", ctypes.POINTER(ctypes.c_double))]


class ie_options(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("max_outer", ctypes.c_int), ("autotune", ctypes.c_int)]


class ie_solve_info(ctypes.Structure):
    _fields_ = [("outer_iters", ctypes.c_int), ("inner_iters", ctypes.c_int),
                ("final_rel_res", ctypes.c_double), ("t_solve", ctypes.c_double),
                ("reorth", ctypes.c_int)]


class IEError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg}: status {status}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load the library (once).  Raises OSError if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"{path} not found: build it with paper_1512_06126_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P, I, D, VP = ctypes.POINTER, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    lib.ie_setup.argtypes = [P(ie_grid), P(ie_layers), P(D), I, P(D), P(D), I, P(ie_options), P(VP)]
    lib.ie_setup.restype = I
    lib.ie_generate_coefficients.argtypes = [P(ie_grid), P(ie_layers), D, VP, VP]
    lib.ie_generate_coefficients.restype = I
    lib.ie_matvec_noalloc.argtypes = [I, I, I, I, VP, VP, VP, VP, VP, VP, VP]
    lib.ie_matvec_noalloc.restype = I
    lib.ie_noalloc_sync.argtypes = [VP]
    lib.ie_noalloc_sync.restype = I
    lib.ie_matvec.argtypes = [VP, I, VP, VP, I, I, I, VP]
    lib.ie_matvec.restype = I
    lib.ie_sync.argtypes = [VP, VP]
    lib.ie_sync.restype = I
    lib.ie_fields.argtypes = [VP, VP, VP, I, VP]
    lib.ie_fields.restype = I
    lib.ie_debug_set_wait_limit.argtypes = [ctypes.c_longlong]
    lib.ie_debug_set_wait_limit.restype = None
    lib.ie_solve.argtypes = [VP, I, VP, VP, I, D, I, I, P(ie_solve_info)]
    lib.ie_solve.restype = I
    lib.ie_adjoint_solve.argtypes = [VP, I, VP, VP, I, D, I, I, P(ie_solve_info)]
    lib.ie_adjoint_solve.restype = I
    lib.ie_rhs_mt.argtypes = [VP, I, I, VP]
    lib.ie_rhs_mt.restype = I
    lib.ie_solve_batch.argtypes = [VP, I, VP, VP, VP, I, D, I, I, I, P(ie_solve_info)]
    lib.ie_solve_batch.restype = I
    lib.ie_contract_tuning.argtypes = [VP, VP, VP]
    lib.ie_contract_tuning.restype = I
    lib.ie_fft_plan.argtypes = [VP, I, VP, VP, VP]
    lib.ie_fft_plan.restype = I
    lib.ie_set_fft_plan.argtypes = [VP, I, VP, I]
    lib.ie_set_fft_plan.restype = I
    lib.ie_set_contract_variant.argtypes = [VP, I, I]
    lib.ie_set_contract_variant.restype = I
    lib.ie_set_sigma.argtypes = [VP, VP]
    lib.ie_set_sigma.restype = I
    lib.ie_set_receivers.argtypes = [VP, I, VP, VP, D]
    lib.ie_set_receivers.restype = I
    lib.ie_set_receivers_xy.argtypes = [VP, I, VP, VP, D]
    lib.ie_set_receivers_xy.restype = I
    lib.ie_mt_apparent.argtypes = [VP, I, VP, I, VP, VP]
    lib.ie_mt_apparent.restype = I
    lib.ie_receiver_fields.argtypes = [VP, I, VP, I, VP, VP]
    lib.ie_receiver_fields.restype = I
    lib.ie_mt_misfit.argtypes = [VP, VP, VP, VP, P(D), VP]
    lib.ie_mt_misfit.restype = I
    lib.ie_receiver_adjoint.argtypes = [VP, I, VP, I, VP]
    lib.ie_receiver_adjoint.restype = I
    lib.ie_gradient_accumulate.argtypes = [VP, VP, VP, I, VP]
    lib.ie_gradient_accumulate.restype = I
    lib.ie_ctx_stream.argtypes = [VP]
    lib.ie_ctx_stream.restype = VP
    lib.ie_ctx_device_bytes.argtypes = [VP]
    lib.ie_ctx_device_bytes.restype = ctypes.c_longlong
    lib.ie_profile.argtypes = [VP, I]
    lib.ie_profile.restype = I
    lib.ie_profile_read.argtypes = [VP, I, P(D), P(ctypes.c_longlong)]
    lib.ie_profile_read.restype = I
    lib.ie_profile_matvec.argtypes = [VP, I, I, I, I, P(D)]
    lib.ie_profile_matvec.restype = I
    lib.ie_kernel_launches.argtypes = []
    lib.ie_kernel_launches.restype = ctypes.c_longlong
    lib.ie_destroy.argtypes = [VP]
    lib.ie_destroy.restype = None
    lib.ie_status_str.argtypes = [I]
    lib.ie_status_str.restype = ctypes.c_char_p
    _lib = lib
    return lib


def kernel_launches() -> int:
    return int(load().ie_kernel_launches())


def matvec_noalloc(nx, ny, nz, nrhs, qf_ptr, in_scale_ptr, out_scale_ptr, diag_ptr, x_ptr, y_ptr, stream=None):
    """Allocation-free c64 product (see ie_matvec_noalloc in include/ie.h).  Returns the
    status code (IE_OK, or IE_ERR_SCRATCH for a problem above the fixed work space)."""
    return load().ie_matvec_noalloc(nx, ny, nz, nrhs, qf_ptr, in_scale_ptr, out_scale_ptr, diag_ptr, x_ptr, y_ptr,
                                    stream)


def noalloc_sync(stream=None):
    """Wait for the stream; IE_ERR_TIMEOUT if a contraction of ie_matvec_noalloc ran out of
    a bounded wait since the last call, else IE_OK."""
    return load().ie_noalloc_sync(stream)


def debug_set_wait_limit(polls: int):
    """Testing aid: polls before the main waits of later contraction launches give up
    (0: at once; negative: the default)."""
    load().ie_debug_set_wait_limit(int(polls))


def status_str(s: int) -> str:
    return load().ie_status_str(s).decode()


def _check(s, what, ok=(IE_OK,)):
    if s not in ok:
        raise IEError(s, f"{what} failed ({status_str(s)})")
    return s


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _cplx_pairs(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128)).view(np.float64)


def _grid_layers(grid, layers, keep):
    ze = np.ascontiguousarray(np.asarray(grid.z_edges, dtype=np.float64))
    d = np.ascontiguousarray(np.asarray(layers.interfaces, dtype=np.float64))
    sig = _cplx_pairs(layers.sigma)
    keep += [ze, d, sig]
    return (ie_grid(grid.nx, grid.ny, grid.nz, grid.hx, grid.hy, _dptr(ze), 0.0, 0.0),
            ie_layers(len(d), _dptr(d), _dptr(sig)))


def generate_coefficients(grid, layers, freq, q_ptr, stream=None):
    """Compressed real-space tensor [Ny][Nx][6][Nz][Nz] (c128) written to the device
    buffer q_ptr by the library's generator."""
    keep = []
    g, lay = _grid_layers(grid, layers, keep)
    _check(load().ie_generate_coefficients(ctypes.byref(g), ctypes.byref(lay), float(freq), q_ptr, stream),
           "ie_generate_coefficients")


class Context:
    """Owns one ie_ctx.  ``q_real`` is a list (one per frequency) of compressed
    real-space tensors [Ny][Nx][6][Nz][Nz] (complex), or None to let the library
    generate them on the device."""

    def __init__(self, grid, layers, sigma_a, freqs, q_real, max_rhs=2, restart=30, max_iter=2000,
                 inner_tol=1e-3, max_outer=50, autotune=True):
        lib = load()
        self._lib = lib
        self._keep = []
        ze = np.ascontiguousarray(np.asarray(grid.z_edges, dtype=np.float64))
        g = ie_grid(grid.nx, grid.ny, grid.nz, grid.hx, grid.hy, _dptr(ze), 0.0, 0.0)
        d = np.ascontiguousarray(np.asarray(layers.interfaces, dtype=np.float64))
        sig = _cplx_pairs(layers.sigma)
        lay = ie_layers(len(d), _dptr(d), _dptr(sig))
        sa = _cplx_pairs(np.asarray(sigma_a).reshape(-1))
        fr = np.ascontiguousarray(np.asarray(freqs, dtype=np.float64))
        if q_real is None:
            q = None
        else:
            q = _cplx_pairs(np.stack([np.asarray(x, dtype=np.complex128) for x in q_real]).reshape(-1))
        opt = ie_options(restart, max_iter, inner_tol, max_outer, 1 if autotune else -1)
        ctx = ctypes.c_void_p()
        s = lib.ie_setup(ctypes.byref(g), ctypes.byref(lay), _dptr(sa), len(fr), _dptr(fr),
                         None if q is None else _dptr(q), max_rhs,
                         ctypes.byref(opt), ctypes.byref(ctx))
        _check(s, "ie_setup")
        self.ctx = ctx
        self.grid = grid
        self.max_rhs = max_rhs
        self.n_unknowns = 3 * grid.nx * grid.ny * grid.nz
        self.n_instances = len(fr)

    def close(self):
        if getattr(self, "ctx", None):
            self._lib.ie_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def stream(self):
        return self._lib.ie_ctx_stream(self.ctx)

    def device_bytes(self):
        return int(self._lib.ie_ctx_device_bytes(self.ctx))

    def matvec(self, inst, x_ptr, y_ptr, nrhs, dtype=IE_C128, transpose=False, stream=None):
        s = self._lib.ie_matvec(self.ctx, inst, x_ptr, y_ptr, nrhs, dtype, int(bool(transpose)), stream)
        _check(s, "ie_matvec")

    def sync(self, stream=None):
        """Wait for the stream (None: the context stream); returns IE_OK or IE_ERR_TIMEOUT."""
        return self._lib.ie_sync(self.ctx, stream)

    def fields(self, u_ptr, e_ptr, nrhs, stream=None):
        """E = U / a for nrhs c128 solutions (asynchronous)."""
        _check(self._lib.ie_fields(self.ctx, u_ptr, e_ptr, nrhs, stream), "ie_fields")

    def solve(self, inst, b_ptr, u_ptr, nrhs, tol, precision=IE_FP64, use_x0=False, adjoint=False):
        info = ie_solve_info()
        fn = self._lib.ie_adjoint_solve if adjoint else self._lib.ie_solve
        s = fn(self.ctx, inst, b_ptr, u_ptr, nrhs, tol, precision, int(bool(use_x0)), ctypes.byref(info))
        _check(s, "ie_adjoint_solve" if adjoint else "ie_solve", ok=(IE_OK, IE_NOT_CONVERGED, IE_BREAKDOWN))
        return s, info

    def solve_batch(self, insts, b_ptr, u_ptr, nrhs, tol, precision=IE_FP64, use_x0=False, adjoint=False):
        """Solve the instances ``insts`` together (vectors [len(insts)][nrhs][3][Nz][Ny][Nx])."""
        ia = np.ascontiguousarray(np.asarray(insts, dtype=np.int32))
        info = ie_solve_info()
        s = self._lib.ie_solve_batch(self.ctx, int(ia.size), ia.ctypes.data, b_ptr, u_ptr, nrhs, tol, precision,
                                     int(bool(use_x0)), int(bool(adjoint)), ctypes.byref(info))
        _check(s, "ie_solve_batch", ok=(IE_OK, IE_NOT_CONVERGED, IE_BREAKDOWN))
        return s, info

    def contract_tuning(self):
        """(variants for 1..4 right-hand sides per instance, autotuner ms [4][N_CONTRACT_VARIANTS])."""
        v = np.zeros(4, dtype=np.int32)
        ms = np.zeros((4, N_CONTRACT_VARIANTS), dtype=np.float64)
        _check(self._lib.ie_contract_tuning(self.ctx, v.ctypes.data, ms.ctypes.data), "ie_contract_tuning")
        return v, ms

    def fft_plan(self, axis):
        """(radices of the FFT plan of axis 0 (x) or 1 (y), ms per c128 pass or 0)."""
        r = np.zeros(20, dtype=np.int32)
        n = ctypes.c_int(0)
        ms = ctypes.c_double(0.0)
        _check(self._lib.ie_fft_plan(self.ctx, axis, r.ctypes.data, ctypes.addressof(n), ctypes.addressof(ms)),
               "ie_fft_plan")
        return [int(v) for v in r[:n.value]], ms.value

    def set_fft_plan(self, axis, radices):
        r = np.ascontiguousarray(radices, dtype=np.int32)
        _check(self._lib.ie_set_fft_plan(self.ctx, axis, r.ctypes.data, len(r)), "ie_set_fft_plan")

    def set_contract_variant(self, nrhs, variant):
        _check(self._lib.ie_set_contract_variant(self.ctx, nrhs, variant), "ie_set_contract_variant")

    def profile(self, enable):
        """0/False off, 1/True the contraction launches, 2 also the steps of every Krylov
        iteration."""
        _check(self._lib.ie_profile(self.ctx, int(enable)), "ie_profile")

    def profile_read(self, dtype):
        ms = ctypes.c_double()
        n = ctypes.c_longlong()
        _check(self._lib.ie_profile_read(self.ctx, dtype, ctypes.byref(ms), ctypes.byref(n)), "ie_profile_read")
        return ms.value, n.value

    def profile_matvec(self, inst, nrhs, dtype, n_iter):
        out = (ctypes.c_double * 5)()
        _check(self._lib.ie_profile_matvec(self.ctx, inst, nrhs, dtype, n_iter, out), "ie_profile_matvec")
        return list(out)

    def rhs_mt(self, inst, pol, u0_ptr):
        _check(self._lib.ie_rhs_mt(self.ctx, inst, pol, u0_ptr), "ie_rhs_mt")

    def set_sigma(self, sigma_a):
        """New anomaly conductivities [Nz][Ny][Nx] (complex) without new coefficients."""
        sa = _cplx_pairs(np.asarray(sigma_a).reshape(-1))
        _check(self._lib.ie_set_sigma(self.ctx, _dptr(sa)), "ie_set_sigma")

    def set_receivers(self, ix, iy, z_rec=0.0):
        ix = np.ascontiguousarray(np.asarray(ix, dtype=np.int32))
        iy = np.ascontiguousarray(np.asarray(iy, dtype=np.int32))
        if ix.shape != iy.shape:
            raise ValueError("ix and iy differ in length")
        _check(self._lib.ie_set_receivers(self.ctx, int(ix.size), ix.ctypes.data, iy.ctypes.data, float(z_rec)),
               "ie_set_receivers")
        self.n_rec = int(ix.size)

    def set_receivers_xy(self, x, y, z_rec=0.0):
        """Receivers at arbitrary lateral sites (metres, the grid's frame)."""
        x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
        y = np.ascontiguousarray(np.asarray(y, dtype=np.float64))
        if x.shape != y.shape:
            raise ValueError("x and y differ in length")
        _check(self._lib.ie_set_receivers_xy(self.ctx, int(x.size), x.ctypes.data, y.ctypes.data, float(z_rec)),
               "ie_set_receivers_xy")
        self.n_rec = int(x.size)

    def mt_apparent(self, inst, z_ptr, n_rec, rho_ptr, phase_ptr):
        """Apparent resistivity and phase [n_rec][4] (FP64, device) from impedances [n_rec][4]."""
        _check(self._lib.ie_mt_apparent(self.ctx, inst, z_ptr, n_rec, rho_ptr, phase_ptr), "ie_mt_apparent")

    def receiver_fields(self, inst, u_ptr, nrhs, pols, f_ptr):
        pa = np.ascontiguousarray(np.asarray(pols, dtype=np.int32))
        _check(self._lib.ie_receiver_fields(self.ctx, inst, u_ptr, nrhs, pa.ctypes.data, f_ptr), "ie_receiver_fields")

    def mt_misfit(self, f_ptr, zobs_ptr, z_ptr, c_ptr):
        phi = ctypes.c_double()
        _check(self._lib.ie_mt_misfit(self.ctx, f_ptr, zobs_ptr, z_ptr, ctypes.byref(phi), c_ptr), "ie_mt_misfit")
        return phi.value

    def receiver_adjoint(self, inst, c_ptr, nrhs, rhs_ptr):
        _check(self._lib.ie_receiver_adjoint(self.ctx, inst, c_ptr, nrhs, rhs_ptr), "ie_receiver_adjoint")

    def gradient_accumulate(self, u_ptr, w_ptr, nrhs, grad_ptr):
        _check(self._lib.ie_gradient_accumulate(self.ctx, u_ptr, w_ptr, nrhs, grad_ptr), "ie_gradient_accumulate")
