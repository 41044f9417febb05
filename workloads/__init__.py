"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the integral-equation method: it only
draws grids, layer stacks, anomaly conductivities, frequencies, random vectors
and random coefficient tensors from fixed seeds.  Everything that computes a
Green's tensor, a coefficient, an operator or a solution lives elsewhere.

Conventions (SI units, time dependence e^{-i omega t}, z positive downwards,
the earth surface at z = 0 and the air above it):

* ``Grid``: ``nx * ny * nz`` cells of ``hx * hy`` laterally; ``z_edges`` holds
  the ``nz + 1`` increasing cell boundaries in metres.
* ``Layers``: ``interfaces[0..L-1]`` = d_1 .. d_L (d_1 = 0 is the surface);
  ``sigma[0..L]`` = air sigma_0, finite layers sigma_1 .. sigma_{L-1} and the
  basement sigma_L, in S/m.
* Cell arrays are ordered ``[z][y][x]``.
* A compressed real-space coefficient tensor (the layout of the operator's
  symmetry-compressed storage, Sect. 3.1) is a complex array
  ``[Ny][Nx][6][Nz][Nz]`` with block order xx, yy, zz, xy, xz, yz for the
  lateral offsets i in [0, Ny), j in [0, Nx).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BLOCKS = ("xx", "yy", "zz", "xy", "xz", "yz")
AIR_SIGMA = 1e-10


@dataclasses.dataclass(frozen=True)
class Grid:
    nx: int
    ny: int
    nz: int
    hx: float
    hy: float
    z_edges: tuple

    @property
    def n_cells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_unknowns(self) -> int:
        return 3 * self.n_cells

    def z_edges_array(self) -> np.ndarray:
        return np.asarray(self.z_edges, dtype=np.float64)


@dataclasses.dataclass(frozen=True)
class Layers:
    interfaces: tuple  # d_1 .. d_L
    sigma: tuple       # sigma_0 .. sigma_L (complex allowed)

    def interfaces_array(self) -> np.ndarray:
        return np.asarray(self.interfaces, dtype=np.float64)

    def sigma_array(self) -> np.ndarray:
        return np.asarray(self.sigma, dtype=np.complex128)


@dataclasses.dataclass(frozen=True)
class Model:
    """One workload instance: grid, background, anomaly, frequencies, sources."""
    name: str
    grid: Grid
    layers: Layers
    sigma_a: np.ndarray          # [nz][ny][nx] complex anomaly conductivity
    freqs: tuple                 # Hz
    pols: tuple                  # subset of ("x", "y")

    @property
    def n_instances(self) -> int:
        return len(self.freqs) * len(self.pols)


def uniform_grid(nx, ny, nz, h, hz=None, z0=0.0) -> Grid:
    hz = h if hz is None else hz
    return Grid(nx, ny, nz, float(h), float(h), tuple(z0 + hz * k for k in range(nz + 1)))


def layer_of(layers: Layers, z: float) -> int:
    """Index of the layer containing depth z (interfaces belong to the lower layer)."""
    d = layers.interfaces
    m = 0
    for k, dk in enumerate(d):
        if z >= dk:
            m = k + 1
    return m


def background_sigma(grid: Grid, layers: Layers) -> np.ndarray:
    """Background conductivity per z-cell (the layer holding the cell centre)."""
    ze = grid.z_edges
    sig = layers.sigma
    return np.array([sig[layer_of(layers, 0.5 * (ze[k] + ze[k + 1]))] for k in range(grid.nz)],
                    dtype=np.complex128)


def _log_uniform(rng, lo, hi, size=None):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=size))


# ----------------------------------------------------------------------------
# The five workloads.  Seeds and recipes are fixed; every array is regenerated
# from them on demand, so no data files are needed.
# ----------------------------------------------------------------------------

def config1() -> Model:
    """8x8x4 cells of 100 m; air / 100 ohm-m 500 m / 10 ohm-m 1500 m / 1000 ohm-m;
    one 4x4x2 block of 0.1 ohm-m; 0.1 Hz; x-polarisation."""
    grid = uniform_grid(8, 8, 4, 100.0)
    layers = Layers((0.0, 500.0, 2000.0), (AIR_SIGMA, 1 / 100.0, 1 / 10.0, 1 / 1000.0))
    sb = background_sigma(grid, layers)
    sa = np.broadcast_to(sb[:, None, None], (4, 8, 8)).astype(np.complex128).copy()
    sa[1:3, 2:6, 2:6] = 1 / 0.1
    return Model("C1", grid, layers, sa, (0.1,), ("x",))


def random_layers(rng, n_layers_total, depth, dz, rho_lo, rho_hi) -> Layers:
    """``n_layers_total`` layers including the basement; interfaces on multiples of dz
    strictly inside (0, depth)."""
    n_int = n_layers_total - 1
    slots = np.arange(1, int(round(depth / dz)))
    cuts = np.sort(rng.choice(slots, size=n_int, replace=False)) * dz
    rho = _log_uniform(rng, rho_lo, rho_hi, size=n_layers_total)
    interfaces = (0.0,) + tuple(float(c) for c in cuts)
    sigma = (AIR_SIGMA,) + tuple(float(1 / r) for r in rho)
    return Layers(interfaces, sigma)


def random_boxes(rng, grid: Grid, sa: np.ndarray, n_boxes, side_xy, side_z, rho_lo, rho_hi):
    """Axis-aligned boxes snapped to cells; later boxes overwrite earlier ones."""
    for _ in range(n_boxes):
        sx = int(rng.integers(side_xy[0], side_xy[1] + 1))
        sy = int(rng.integers(side_xy[0], side_xy[1] + 1))
        sz = int(rng.integers(side_z[0], side_z[1] + 1))
        sx, sy, sz = min(sx, grid.nx), min(sy, grid.ny), min(sz, grid.nz)
        x0 = int(rng.integers(0, grid.nx - sx + 1))
        y0 = int(rng.integers(0, grid.ny - sy + 1))
        z0 = int(rng.integers(0, grid.nz - sz + 1))
        sa[z0:z0 + sz, y0:y0 + sy, x0:x0 + sx] = 1.0 / float(_log_uniform(rng, rho_lo, rho_hi))
    return sa


def _anomalous_model(name, seed, n, nz, h, n_layers, rho_layers, n_boxes, side_xy, side_z, rho_box,
                     freqs, pols) -> Model:
    rng = np.random.default_rng(seed)
    grid = uniform_grid(n, n, nz, h)
    layers = random_layers(rng, n_layers, nz * h, h, *rho_layers)
    sb = background_sigma(grid, layers)
    sa = np.broadcast_to(sb[:, None, None], (nz, n, n)).astype(np.complex128).copy()
    sa = random_boxes(rng, grid, sa, n_boxes, side_xy, side_z, *rho_box)
    return Model(name, grid, layers, sa, tuple(freqs), tuple(pols))


def config2() -> Model:
    """128x128x32 cells of 50 m; 5 layers incl. basement, rho log-U[1,1000] (seed 2);
    20 boxes at 0.01-0.1 ohm-m; 1 Hz; both polarisations."""
    return _anomalous_model("C2", 2, 128, 32, 50.0, 5, (1.0, 1000.0), 20, (4, 24), (2, 8),
                            (0.01, 0.1), (1.0,), ("x", "y"))


def config3() -> list:
    """Four grids (64,16), (96,24), (128,32), (192,48) of 50 m cells (seeds 30-33);
    16 log-spaced frequencies in [1e-3, 1e2] Hz x 2 polarisations; frequency k on grid k mod 4."""
    freqs = np.logspace(-3, 2, 16)
    shapes = [(64, 16), (96, 24), (128, 32), (192, 48)]
    out = []
    for g, (n, nz) in enumerate(shapes):
        fk = tuple(float(f) for k, f in enumerate(freqs) if k % 4 == g)
        out.append(_anomalous_model(f"C3g{g}", 30 + g, n, nz, 50.0, 5, (1.0, 1000.0), 12, (4, max(5, n // 6)),
                                    (2, max(3, nz // 4)), (0.01, 0.1), fk, ("x", "y")))
    return out


def config4() -> Model:
    """64x64x24 cells of 50 m; 3 layers + basement (seed 4); 2 conductive boxes;
    8 frequencies in [1e-2, 1e1] Hz x 2 polarisations."""
    return _anomalous_model("C4", 4, 64, 24, 50.0, 4, (10.0, 1000.0), 2, (8, 20), (3, 8), (0.1, 1.0),
                            tuple(float(f) for f in np.logspace(-2, 1, 8)), ("x", "y"))


def config5() -> Model:
    """256x256x64 cells of 25 m; 8 layers, rho log-U[0.3,3000] (seed 5); 200 boxes at 0.01 ohm-m;
    0.01 Hz; 2 polarisations."""
    return _anomalous_model("C5", 5, 256, 64, 25.0, 8, (0.3, 3000.0), 200, (4, 24), (2, 8),
                            (0.01, 0.01), (0.01,), ("x", "y"))


# The seven blocks of the COMMEMI3D-3 model (Sect. 4, Table (commemi_table)): opposite
# corners (x1, y1, z1), (x2, y2, z2) in km and conductivity in S/m
COMMEMI3D3_BLOCKS = (
    ((0.0, 2.4, 0.05), (3.0, 2.8, 0.30), 0.0033),
    ((0.0, 1.8, 0.05), (3.0, 2.4, 0.45), 0.033),
    ((0.0, 1.4, 0.05), (3.0, 1.8, 0.30), 0.1),
    ((0.0, 0.8, 0.05), (3.0, 1.4, 0.45), 0.033),
    ((0.0, 0.4, 0.05), (3.0, 0.8, 0.30), 0.0033),
    ((3.4, 2.8, 0.20), (4.4, 4.8, 1.00), 10.0),
    ((1.4, 0.0, 1.00), (2.4, 5.6, 3.00), 3.3333),
)
# the model's (x, y) origin in the grid's frame (m): the grid spans x in [-1.0, 5.4] km,
# y in [-0.4, 6.0] km of the model
COMMEMI3D3_ORIGIN = (1000.0, 400.0)


def commemi3d3_like() -> Model:
    """A COMMEMI3D-3-like synthetic model (Sect. 4): the seven blocks of its table in its
    layered background (air; 1e-3 S/m to 1 km; 1e-4 S/m to 7.5 km; 0.1 S/m below) on
    64 x 64 cells of 100 m laterally and 32 cells in z (50 m from 50 to 450 m, 68.75 m to
    1 km, 125 m to 3 km, so that every block face and the interface at 1 km are cell
    faces); a cell takes the conductivity of the block holding its centre; period 1 s,
    both polarisations.  Grid x = model x + 1 km, grid y = model y + 0.4 km."""
    ze = ([50.0 * k for k in range(1, 10)] + [450.0 + 68.75 * k for k in range(1, 9)] +
          [1000.0 + 125.0 * k for k in range(1, 17)])
    grid = Grid(64, 64, 32, 100.0, 100.0, tuple(ze))
    layers = Layers((0.0, 1000.0, 7500.0), (AIR_SIGMA, 1e-3, 1e-4, 0.1))
    sb = background_sigma(grid, layers)
    sa = np.broadcast_to(sb[:, None, None], (grid.nz, grid.ny, grid.nx)).astype(np.complex128).copy()
    zc = 0.5 * (np.asarray(ze[:-1]) + np.asarray(ze[1:]))
    xc = (np.arange(grid.nx) + 0.5) * grid.hx - COMMEMI3D3_ORIGIN[0]
    yc = (np.arange(grid.ny) + 0.5) * grid.hy - COMMEMI3D3_ORIGIN[1]
    for (x1, y1, z1), (x2, y2, z2), sig in COMMEMI3D3_BLOCKS:
        kz = (zc > 1000 * z1) & (zc < 1000 * z2)
        ky = (yc > 1000 * y1) & (yc < 1000 * y2)
        kx = (xc > 1000 * x1) & (xc < 1000 * x2)
        sa[np.ix_(kz, ky, kx)] = sig
    return Model("COMMEMI3D-3-like", grid, layers, sa, (1.0,), ("x", "y"))


def small_model(nx=6, ny=5, nz=3, h=100.0, seed=7, freq=1.0, pols=("x",), n_layers=3) -> Model:
    """A small ragged model for tests: Nx != Ny, several layers crossing the cell column."""
    rng = np.random.default_rng(seed)
    grid = Grid(nx, ny, nz, float(h), float(h) * 1.25,
                tuple(float(v) for v in np.concatenate([[0.0], np.cumsum(h * rng.choice([0.5, 1.0, 1.5], nz))])))
    depth = grid.z_edges[-1]
    # interfaces on cell edges so that no cell straddles one
    cand = list(grid.z_edges[1:-1])
    k = min(n_layers - 1, len(cand))
    cuts = sorted(rng.choice(cand, size=k, replace=False)) if k > 0 else []
    rho = _log_uniform(rng, 3.0, 300.0, size=len(cuts) + 1)
    layers = Layers((0.0,) + tuple(float(c) for c in cuts), (AIR_SIGMA,) + tuple(float(1 / r) for r in rho))
    sb = background_sigma(grid, layers)
    sa = np.broadcast_to(sb[:, None, None], (nz, ny, nx)).astype(np.complex128).copy()
    sa = random_boxes(rng, grid, sa, 2, (1, 3), (1, 2), 0.3, 3.0)
    assert depth > 0
    return Model(f"small{nx}x{ny}x{nz}", grid, layers, sa, (float(freq),), tuple(pols))


# ----------------------------------------------------------------------------
# Random vectors and tensors
# ----------------------------------------------------------------------------

def random_field(shape, seed, dtype=np.complex128) -> np.ndarray:
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return v.astype(dtype)


def random_compressed_q(ny, nx, nz, seed, decay=0.15) -> np.ndarray:
    """Random coefficient tensor in the compressed real-space layout
    ``[Ny][Nx][6][Nz][Nz]`` (xx, yy, zz, xy upper triangles symmetric; xz, yz full).

    Magnitudes fall off with the lateral offset like a smooth envelope so that the
    tensor looks like a decaying kernel; the values carry no physics.  The
    blocks that a lateral parity forces to vanish on the axes (xy at i = 0 or
    j = 0, xz at j = 0, yz at i = 0) are zero there, as in a physical tensor.
    """
    rng = np.random.default_rng(seed)
    q = rng.standard_normal((ny, nx, 6, nz, nz)) + 1j * rng.standard_normal((ny, nx, 6, nz, nz))
    ii, jj = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    env = 1.0 / (1.0 + decay * (ii ** 2 + jj ** 2)) ** 1.5
    q *= env[:, :, None, None, None]
    for b in range(4):  # xx, yy, zz, xy are symmetric in z
        q[:, :, b] = 0.5 * (q[:, :, b] + np.swapaxes(q[:, :, b], -1, -2))
    q[0, :, 3] = 0.0
    q[:, 0, 3] = 0.0
    q[:, 0, 4] = 0.0
    q[0, :, 5] = 0.0
    return q
