"""The system matrix A = S + R1 B R2 and its solution.

Test infrastructure (see ``oracle/__init__``).  Paper: eq. (slae1),
(slae_matricies), (matrix_convolv); the FFT matrix-vector product of Sect. 3.3;
FGMRES of Sect. 3.3 (ii) (here restarted GMRES, classical Gram-Schmidt applied
twice); dense LU for small systems.

Vectors are complex arrays [3][Nz][Ny][Nx] (component x, y, z; x fastest).

  (A U)_n = U_n - sum_m gamma_m K_n^m U_m,   K_n^m = delta_nm I + (2/V_n) s_n s_m B_n^m,
  gamma_m = (sigma_a - sigma_b) / (sigma_a + conj(sigma_b)),  s = sqrt(Re sigma_b),

so A = S + R1 B R2 with S = diag(1 - gamma), R1 = -diag(2 s / V), R2 = diag(s gamma).

Parity: the dense apply is pinned by the FFT apply (two independent routes:
brute-force negative offsets vs. the 2N-periodic embedding with the lateral
parities), by sigma_a = sigma_b => U = U^0, by the contraction bound of the
modified operator (Sect. 2.1) and by dense LU = GMRES (uniqueness, Sect. 2.2).
"""
from __future__ import annotations

import numpy as np

from workloads import background_sigma
from .coefficients import full_block

# lateral parities (sign under x -> -x, sign under y -> -y) of xx, yy, zz, xy, xz, yz
PARITY = ((1, 1), (1, 1), (1, 1), (-1, -1), (-1, 1), (1, -1))


def diagonals(model):
    """gamma [Nz][Ny][Nx], s [Nz] (per z-cell) and the cell volumes V [Nz]."""
    g = model.grid
    sb = background_sigma(g, model.layers)
    sa = np.asarray(model.sigma_a, dtype=np.complex128)
    gamma = (sa - sb[:, None, None]) / (sa + np.conj(sb)[:, None, None])
    s = np.sqrt(sb.real)
    V = g.hx * g.hy * np.diff(g.z_edges_array())
    return gamma, s, V


def in_cell_field(model, U):
    """E_n = U_n / a_n with a_n = (sigma_a^n + conj sigma_b^n) / (2 s_n): the change of
    variables under eq. (iEH320op) undone.  U: [R][3][Nz][Ny][Nx] or [3][Nz][Ny][Nx].
    Pinned by sigma_a = sigma_b (E = the cell average of the normal field) and by the
    scattering current (sigma_a - sigma_b) E = 2 s gamma U of eq. (APR_lab) (tests)."""
    g = model.grid
    sb = background_sigma(g, model.layers)
    sa = np.asarray(model.sigma_a, dtype=np.complex128)
    s = np.sqrt(sb.real)
    a = (sa + np.conj(sb)[:, None, None]) / (2.0 * s[:, None, None])
    return np.asarray(U) / a


def dense_B(model, q_all):
    """Brute-force 3N x 3N matrix of the blocks B_n^m from their values at every signed
    offset (q_all as returned by coefficients.all_offsets; no symmetry is used)."""
    g = model.grid
    nx, ny, nz = g.nx, g.ny, g.nz
    N = nx * ny * nz
    B = np.zeros((3 * N, 3 * N), dtype=np.complex128)

    def idx(c, z, y, x):
        return ((c * nz + z) * ny + y) * nx + x
    cz = np.arange(nz)
    for yn in range(ny):
        for xn in range(nx):
            for ym in range(ny):
                for xm in range(nx):
                    blk = full_block(q_all[yn - ym + ny - 1, xn - xm + nx - 1])
                    for cn in range(3):
                        rows = idx(cn, cz, yn, xn)
                        for cm in range(3):
                            cols = idx(cm, cz, ym, xm)
                            B[np.ix_(rows, cols)] = blk[cn * nz:(cn + 1) * nz, cm * nz:(cm + 1) * nz]
    return B


def _per_unknown(model):
    g = model.grid
    gamma, s, V = diagonals(model)
    sN = np.tile(np.broadcast_to(s[:, None, None], gamma.shape).ravel(), 3)
    VN = np.tile(np.broadcast_to(V[:, None, None], gamma.shape).ravel(), 3)
    gN = np.tile(gamma.ravel(), 3)
    return gN, sN, VN


def dense_matrix(model, B):
    """A = diag(1 - gamma) - diag(2 s / V) B diag(s gamma)."""
    gN, sN, VN = _per_unknown(model)
    return np.diag(1.0 - gN) - (2.0 * sN / VN)[:, None] * B * (sN * gN)[None, :]


def dense_K(model, B):
    """The modified operator K = I + diag(2 s / V) B diag(s) of (slae_matricies)."""
    gN, sN, VN = _per_unknown(model)
    return np.eye(B.shape[0]) + (2.0 * sN / VN)[:, None] * B * sN[None, :]


def contraction_norm(model, B):
    """|| V^{1/2} K V^{-1/2} ||_2: the norm of K in L2 (eq. (L_defininition)) for the
    piecewise-constant basis; the Galerkin projection of the contracting operator
    of (Grmod) keeps it at most 1."""
    gN, sN, VN = _per_unknown(model)
    K = dense_K(model, B)
    W = np.sqrt(VN)
    return np.linalg.norm(W[:, None] * K / W[None, :], 2)


def embed_spectrum(q):
    """DFT over the 2N-periodic embedding of the compressed tensor.

    q: [Ny][Nx][6][Nz][Nz] for offsets i in [0,Ny), j in [0,Nx).  The embedding
    puts Q(i, j) at (i mod 2Ny, j mod 2Nx) for |i| < Ny, |j| < Nx, with negative
    offsets from the lateral parities of Lemma 2 and zero at i = Ny or j = Nx.
    Returns the spectrum of the six blocks, [2Ny][2Nx][6][Nz][Nz]."""
    ny, nx, _, nz, _ = q.shape
    emb = np.zeros((2 * ny, 2 * nx, 6, nz, nz), dtype=np.complex128)
    for b, (px, py) in enumerate(PARITY):
        blk = q[:, :, b]
        emb[:ny, :nx, b] = blk
        emb[ny + 1:, :nx, b] = py * blk[1:][::-1]
        emb[:ny, nx + 1:, b] = px * blk[:, 1:][:, ::-1]
        emb[ny + 1:, nx + 1:, b] = px * py * blk[1:, 1:][::-1, ::-1]
    return np.fft.fft2(emb, axes=(0, 1))


def full_spectrum_blocks(qt):
    """[2Ny][2Nx][3Nz][3Nz] blocks from the six-block spectrum (Lemma 1 for zx, zy)."""
    xx, yy, zz, xy, xz, yz = (qt[:, :, b] for b in range(6))
    T = lambda a: np.swapaxes(a, -1, -2)
    row0 = np.concatenate([xx, xy, xz], -1)
    row1 = np.concatenate([xy, yy, yz], -1)
    row2 = np.concatenate([-T(xz), -T(yz), zz], -1)
    return np.concatenate([row0, row1, row2], -2)


def fft_apply(model, qt_full, x, transpose=False):
    """A x (or A^T x) through the zero-padded 2-D FFT, Sect. 3.3.  x: [3][Nz][Ny][Nx]."""
    g = model.grid
    nx, ny, nz = g.nx, g.ny, g.nz
    gamma, s, V = diagonals(model)
    sg = s[:, None, None] * gamma
    r1 = -(2.0 / V) * s
    if not transpose:
        xin = sg[None] * x
    else:
        xin = r1[None, :, None, None] * x
    pad = np.zeros((3, nz, 2 * ny, 2 * nx), dtype=np.complex128)
    pad[:, :, :ny, :nx] = xin
    spec = np.fft.fft2(pad, axes=(2, 3))                     # [3][Nz][2Ny][2Nx]
    v = spec.reshape(3 * nz, 2 * ny, 2 * nx).transpose(1, 2, 0)   # [2Ny][2Nx][3Nz]
    if transpose:
        # (B^T)_{nm} = (B_{mn})^T: offset -D, i.e. the spectrum Q(-k)^T
        qneg = qt_full[(-np.arange(2 * ny)) % (2 * ny)][:, (-np.arange(2 * nx)) % (2 * nx)]
        w = np.einsum("yxba,yxb->yxa", qneg, v)
    else:
        w = np.einsum("yxab,yxb->yxa", qt_full, v)
    w = w.transpose(2, 0, 1).reshape(3, nz, 2 * ny, 2 * nx)
    bx = np.fft.ifft2(w, axes=(2, 3))[:, :, :ny, :nx]
    if not transpose:
        return (1.0 - gamma)[None] * x + r1[None, :, None, None] * bx
    return (1.0 - gamma)[None] * x + sg[None] * bx


def gmres(apply, b, tol=1e-12, m=30, max_iter=2000, x0=None):
    """Restarted GMRES(m), classical Gram-Schmidt applied twice, FP64.
    Returns (x, n_iter, rel_res_history)."""
    bshape = b.shape
    bv = b.ravel()
    nb = np.linalg.norm(bv)
    x = np.zeros_like(bv) if x0 is None else x0.ravel().copy()
    hist = []
    it = 0
    if nb == 0:
        return x.reshape(bshape), 0, [0.0]
    while it < max_iter:
        r = bv - apply(x.reshape(bshape)).ravel()
        beta = np.linalg.norm(r)
        hist.append(beta / nb)
        if beta / nb <= tol:
            break
        Vb = np.zeros((m + 1, bv.size), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        Vb[0] = r / beta
        k_used = 0
        for k in range(m):
            w = apply(Vb[k].reshape(bshape)).ravel()
            h = Vb[:k + 1].conj() @ w
            w = w - Vb[:k + 1].T @ h
            h2 = Vb[:k + 1].conj() @ w
            w = w - Vb[:k + 1].T @ h2
            H[:k + 1, k] = h + h2
            H[k + 1, k] = np.linalg.norm(w)
            it += 1
            k_used = k + 1
            e1 = np.zeros(k + 2, dtype=np.complex128)
            e1[0] = beta
            y = np.linalg.lstsq(H[:k + 2, :k + 1], e1, rcond=None)[0]
            res = np.linalg.norm(e1 - H[:k + 2, :k + 1] @ y)
            if H[k + 1, k].real == 0 and H[k + 1, k].imag == 0:
                break
            Vb[k + 1] = w / H[k + 1, k]
            if res / nb <= tol * 0.5 or it >= max_iter:
                break
        x = x + Vb[:k_used].T @ y
    return x.reshape(bshape), it, hist


def block_at(q, i, j):
    """The 3Nz x 3Nz block B(i, j) for any signed offset from the compressed tensor
    q [Ny][Nx][6][Nz][Nz], by the lateral parities of Lemma 2 and Lemma 1."""
    ai, aj = abs(i), abs(j)
    six = np.empty_like(q[0, 0])
    for b, (px, py) in enumerate(PARITY):
        s = (py if i < 0 else 1) * (px if j < 0 else 1)
        six[b] = s * q[ai, aj, b]
    return full_block(six)


def direct_rows(model, q, x, cells):
    """(A x) at the listed cells (z, y, x) by direct summation over every source cell;
    returns an array [len(cells)][3].  q: compressed tensor; x: [3][Nz][Ny][Nx]."""
    g = model.grid
    nz, ny, nx = g.nz, g.ny, g.nx
    gamma, s, V = diagonals(model)
    xs = (s[:, None, None] * gamma)[None] * x                      # R2 x
    out = []
    for (zn, yn, xn) in cells:
        acc = np.zeros(3, dtype=np.complex128)
        for yy in range(ny):
            i = yn - yy
            for xx in range(nx):
                j = xn - xx
                B = block_at(q, i, j)
                rows = B[[zn, nz + zn, 2 * nz + zn]]                  # [3][3Nz]
                acc += rows @ xs[:, :, yy, xx].reshape(-1)
        r1 = -(2.0 / V[zn]) * s[zn]
        out.append((1.0 - gamma[zn, yn, xn]) * x[:, zn, yn, xn] + r1 * acc)
    return np.array(out)
