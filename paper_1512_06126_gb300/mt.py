"""Magnetotelluric impedance misfit and its gradient in ln(sigma_a), behind a
torch.autograd.Function.

Every step runs in the library (ctypes calls of include/ie.h); this module only
sequences them and keeps the device buffers:

  forward, per frequency:  U^0 for both plane-wave polarisations (ie_rhs_mt), the
    solve A U = U^0 (ie_solve, both polarisations in lockstep), the fields at the
    receivers (ie_receiver_fields), Z = E H^-1, the misfit and its adjoint sources
    (ie_mt_misfit);
  backward, per frequency:  the adjoint right-hand side 2 s gamma G^T c
    (ie_receiver_adjoint), the transposed solve A^T w = rhs (ie_adjoint_solve), and
    grad += Re (dgamma/dln sigma_a)(w . U)/gamma (ie_gradient_accumulate).

The Krylov bases are never kept between the passes.  The forward solutions U are
kept for the backward pass (one c128 field pair per frequency); with
``store_fields=False`` they are recomputed by a second forward solve instead, which
trades two solves per frequency for the memory of the stored fields.
"""
from __future__ import annotations

import numpy as np
import torch

from . import ie


class MTProblem:
    """MT misfit Phi = 1/2 sum_{f, r, ij} |Z_ij - Zobs_ij|^2 over the context's
    instances (one frequency each) and the receivers.

    ctx: ie.Context whose instances are the frequencies; receivers: (ix, iy) cell
    columns; zobs: array [n_freq][n_rec][2][2] complex; tol/precision: of the
    forward and adjoint solves."""

    def __init__(self, ctx, ix, iy, zobs, z_rec=0.0, tol=1e-10, precision=ie.IE_FP64, store_fields=True):
        self.ctx = ctx
        g = ctx.grid
        self.shape = (g.nz, g.ny, g.nx)
        ctx.set_receivers(ix, iy, z_rec)
        self.n_rec = len(ix)
        self.n_inst = ctx.n_instances
        zobs = np.asarray(zobs, dtype=np.complex128)
        if zobs.shape != (self.n_inst, self.n_rec, 2, 2):
            raise ValueError(f"zobs must have shape {(self.n_inst, self.n_rec, 2, 2)}")
        dev = torch.device("cuda")
        self.zobs = torch.from_numpy(zobs.copy()).to(dev)
        vshape = (2, 3) + self.shape
        self.b = torch.empty(vshape, dtype=torch.complex128, device=dev)
        self.w = torch.empty_like(self.b)
        self.rhs = torch.empty_like(self.b)
        self.f = torch.empty((2, self.n_rec, 4), dtype=torch.complex128, device=dev)
        self.z = torch.empty((self.n_inst, self.n_rec, 2, 2), dtype=torch.complex128, device=dev)
        self.c = torch.empty((self.n_inst, 2, self.n_rec, 4), dtype=torch.complex128, device=dev)
        self.grad = torch.zeros(self.shape, dtype=torch.float64, device=dev)
        self.store = store_fields
        self.u = [torch.zeros(vshape, dtype=torch.complex128, device=dev) for _ in range(self.n_inst if store_fields else 1)]
        self.tol, self.precision = tol, precision
        self.iters = {"forward": 0, "adjoint": 0}

    def _forward_solve(self, k, u):
        for p in range(2):
            self.ctx.rhs_mt(k, p, self.b[p].data_ptr())
        u.zero_()
        torch.cuda.synchronize()
        st, info = self.ctx.solve(k, self.b.data_ptr(), u.data_ptr(), 2, self.tol, precision=self.precision)
        if st != ie.IE_OK:
            raise RuntimeError(f"forward solve of instance {k}: status {st}, residual {info.final_rel_res:.2e}")
        self.iters["forward"] += info.inner_iters

    def misfit(self) -> float:
        phi = 0.0
        for k in range(self.n_inst):
            u = self.u[k if self.store else 0]
            self._forward_solve(k, u)
            self.ctx.receiver_fields(k, u.data_ptr(), 2, (0, 1), self.f.data_ptr())
            phi += self.ctx.mt_misfit(self.f.data_ptr(), self.zobs[k].data_ptr(), self.z[k].data_ptr(),
                                      self.c[k].data_ptr())
        return phi

    def gradient(self) -> torch.Tensor:
        """dPhi/dln(sigma_a) [Nz][Ny][Nx] on the device (zero off the anomaly), for the
        conductivities of the last ``misfit`` call."""
        self.grad.zero_()
        for k in range(self.n_inst):
            u = self.u[k] if self.store else self.u[0]
            if not self.store:
                self._forward_solve(k, u)
            self.ctx.receiver_adjoint(k, self.c[k].data_ptr(), 2, self.rhs.data_ptr())
            self.w.zero_()
            torch.cuda.synchronize()
            st, info = self.ctx.solve(k, self.rhs.data_ptr(), self.w.data_ptr(), 2, self.tol,
                                      precision=self.precision, adjoint=True)
            if st != ie.IE_OK:
                raise RuntimeError(f"adjoint solve of instance {k}: status {st}, residual {info.final_rel_res:.2e}")
            self.iters["adjoint"] += info.inner_iters
            self.ctx.gradient_accumulate(u.data_ptr(), self.w.data_ptr(), 2, self.grad.data_ptr())
        return self.grad


class MTMisfit(torch.autograd.Function):
    """Phi(theta) for theta = ln(sigma_a) of the cells ``cells`` (flat indices into
    [Nz][Ny][Nx]); the other cells keep ``sigma_base``.  backward gives dPhi/dtheta
    from one adjoint solve per frequency."""

    @staticmethod
    def forward(ctx_, theta, problem, cells, sigma_base):
        sig = np.array(sigma_base, dtype=np.complex128).reshape(-1)
        sig[cells] = np.exp(theta.detach().cpu().numpy())
        problem.ctx.set_sigma(sig.reshape(problem.shape))
        phi = problem.misfit()
        ctx_.problem = problem
        ctx_.cells = torch.as_tensor(np.asarray(cells), device="cuda")
        ctx_.theta_device = theta.device
        return torch.tensor(phi, dtype=torch.float64, device=theta.device)

    @staticmethod
    def backward(ctx_, grad_out):
        g = ctx_.problem.gradient().reshape(-1)[ctx_.cells]
        return grad_out * g.to(ctx_.theta_device), None, None, None
