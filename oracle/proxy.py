"""Synthetic operators of full workload size whose solves the oracle can check.

Test infrastructure (see ``oracle/__init__``): used by tests/ and by the CPU-baseline
leg of bench.py only.

The oracle cannot compute the physical coefficient tensors of the large grids in a
test's time, so the kernels and solvers are checked at those sizes on a proxy: the
workload's grid and layers, the anomalous cells at a moderate contrast, and a seeded
random coefficient tensor (workloads.random_compressed_q) scaled with the oracle's
own diagonals so that A = S + R1 B R2 = (I + E) S with ||E|| <= target.  GMRES then
converges in a few dozen iterations and the answer is unique, so the residual of a
GPU solution under the oracle's FFT product is a meaningful check of every kernel on
the path (FFTs, contraction, scalings, Gram-Schmidt, rotations, refinement)."""
import numpy as np

import workloads as W
from oracle import operator as O


def moderate_contrast(model, factor=3.0):
    """The model with sigma_a = factor * sigma_b wherever it had an anomaly."""
    g = model.grid
    sb = W.background_sigma(g, model.layers)
    base = np.broadcast_to(sb[:, None, None], model.sigma_a.shape)
    sa = np.where(np.abs(model.sigma_a - base) > 0, factor * base, base).astype(np.complex128)
    return W.Model(model.name + "-moderate", g, model.layers, sa, model.freqs, model.pols)


def contracting_q(model, seed, target=0.5, decay=0.15):
    """(q, qt_full): a seeded random compressed tensor scaled so that
    max|R1| max|R2 S^-1| max_k ||Q~(k)||_F = target, and its full spectral blocks for
    oracle.operator.fft_apply."""
    g = model.grid
    q = W.random_compressed_q(g.ny, g.nx, g.nz, seed=seed, decay=decay)
    qt6 = O.embed_spectrum(q)
    w = np.array([1.0, 1.0, 1.0, 2.0, 2.0, 2.0])
    fro = np.sqrt(np.einsum("yxbij,b->yx", np.abs(qt6) ** 2, w)).max()
    gamma, s, V = O.diagonals(model)
    r1 = np.abs(2.0 * s / V).max()
    r2s = np.abs(s[:, None, None] * gamma / (1.0 - gamma)).max()
    scale = target / (r1 * r2s * fro)
    q *= scale
    qt6 *= scale
    qt = O.full_spectrum_blocks(qt6)
    del qt6
    return q, qt


def oracle_residual(model, qt, b, u):
    """max over right-hand sides of ||b - A u|| / ||b|| with the oracle's FFT product."""
    out = 0.0
    for r in range(b.shape[0]):
        res = b[r] - O.fft_apply(model, qt, u[r])
        out = max(out, float(np.linalg.norm(res) / np.linalg.norm(b[r])))
    return out
