"""Cross-well travel-time tomography workloads (Sec. 4.1.1, Eq. lineartomography).

Geometry: the unit square (or cube) is divided into equal cells; the state is
one slowness value per cell, located at the cell centre.  Sources sit on the
x=0 edge (face), receivers on the x=1 edge (face); every source-receiver pair
is one straight ray and one measurement.  Row j of the measurement operator H
holds, for every cell, the length of ray j inside that cell, so that H s is the
travel time of a piecewise-constant slowness s.

The paper's own data (a reservoir simulation) is not available; the truth used
here is a seeded random walk whose increments are smooth Gaussian random fields
made by periodic Gaussian smoothing of white noise.  That smoothing is a
generator choice only -- it is not the filter's Matern covariance.

Index conventions: 2D cell (ix, iy) has index iy*nx + ix; 3D voxel (ix, iy, iz)
has index (iz*ny + iy)*nx + ix.  Ray index = source_index * n_receivers +
receiver_index.
"""

from __future__ import annotations

from dataclasses import dataclass
from typing import Sequence

import numpy as np

BASE_SEED = 14052276


@dataclass
class Csr:
    """A sparse m x N matrix in compressed-row form (int64 rowptr, int32 col)."""

    rowptr: np.ndarray  # int64, m+1
    col: np.ndarray  # int32, nnz (sorted within each row)
    val: np.ndarray  # float64, nnz
    ncols: int

    @property
    def nrows(self) -> int:
        return int(self.rowptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])


def csr_to_dense(h: Csr) -> np.ndarray:
    out = np.zeros((h.nrows, h.ncols))
    for i in range(h.nrows):
        a, b = h.rowptr[i], h.rowptr[i + 1]
        out[i, h.col[a:b]] += h.val[a:b]
    return out


# ----------------------------------------------------------------------------
# points and acquisition geometry
# ----------------------------------------------------------------------------
def grid_points_2d(nx: int, ny: int) -> np.ndarray:
    """Cell centres of an nx x ny grid on [0,1]^2, shape (nx*ny, 2)."""
    ix = (np.arange(nx) + 0.5) / nx
    iy = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(ix, iy, indexing="xy")  # Y varies along axis 0
    return np.stack([X.ravel(), Y.ravel()], axis=1)


def grid_points_3d(nx: int, ny: int, nz: int) -> np.ndarray:
    """Voxel centres of an nx x ny x nz grid on [0,1]^3, shape (N, 3)."""
    gx = (np.arange(nx) + 0.5) / nx
    gy = (np.arange(ny) + 0.5) / ny
    gz = (np.arange(nz) + 0.5) / nz
    Z, Y, X = np.meshgrid(gz, gy, gx, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def cross_well_geometry_2d(n_src: int, n_rec: int):
    """Sources at (0, (a+1/2)/n_src), receivers at (1, (b+1/2)/n_rec)."""
    src = np.stack([np.zeros(n_src), (np.arange(n_src) + 0.5) / n_src], axis=1)
    rec = np.stack([np.ones(n_rec), (np.arange(n_rec) + 0.5) / n_rec], axis=1)
    p0 = np.repeat(src, n_rec, axis=0)
    p1 = np.tile(rec, (n_src, 1))
    return p0, p1


def cross_well_geometry_3d(src_grid: Sequence[int], rec_grid: Sequence[int]):
    """Sources on a (sa x sb) lattice of the x=0 face, receivers on an
    (ra x rb) lattice of the x=1 face; lattice points at (i+1/2)/n."""

    def face(na, nb, x):
        a = (np.arange(na) + 0.5) / na
        b = (np.arange(nb) + 0.5) / nb
        A, B = np.meshgrid(a, b, indexing="ij")
        return np.stack([np.full(A.size, x), A.ravel(), B.ravel()], axis=1)

    src = face(src_grid[0], src_grid[1], 0.0)
    rec = face(rec_grid[0], rec_grid[1], 1.0)
    p0 = np.repeat(src, rec.shape[0], axis=0)
    p1 = np.tile(rec, (src.shape[0], 1))
    return p0, p1


# ----------------------------------------------------------------------------
# straight-ray tracing (parametric crossings with the grid planes)
# ----------------------------------------------------------------------------
def _trace_one(p0, p1, dims, tie_tol=1e-12, grid_tol=1e-9):
    """Cells crossed by the segment p0->p1 and the length inside each.

    The crossing parameters with every grid plane are merged (ties within
    tie_tol become one); each sub-segment is assigned to the cell containing
    its midpoint.  A sub-segment lying exactly in a grid plane is shared
    equally by the cells on both sides of that plane (only those inside the
    domain).
    """
    dim = len(dims)
    d = p1 - p0
    length = float(np.sqrt(np.sum(d * d)))
    ts = [np.array([0.0, 1.0])]
    for ax in range(dim):
        if d[ax] != 0.0:
            planes = np.arange(dims[ax] + 1) / dims[ax]
            t = (planes - p0[ax]) / d[ax]
            ts.append(t[(t > 0.0) & (t < 1.0)])
    t = np.sort(np.concatenate(ts))
    keep = np.concatenate([[True], np.diff(t) > tie_tol])
    t = t[keep]
    if t[-1] < 1.0 - tie_tol:
        t = np.append(t, 1.0)
    t[-1] = 1.0
    tm = 0.5 * (t[:-1] + t[1:])
    seg = np.diff(t) * length
    mids = p0[None, :] + tm[:, None] * d[None, :]
    cells = []
    weights = []
    for k in range(tm.shape[0]):
        choices = []
        for ax in range(dim):
            f = mids[k, ax] * dims[ax]
            fr = np.rint(f)
            if d[ax] == 0.0 and abs(f - fr) < grid_tol:
                c = [int(fr) - 1, int(fr)]
                c = [v for v in c if 0 <= v < dims[ax]]
            else:
                c = [min(max(int(np.floor(f)), 0), dims[ax] - 1)]
            choices.append(c)
        combos = [[]]
        for c in choices:
            combos = [a + [v] for a in combos for v in c]
        w = seg[k] / len(combos)
        for cb in combos:
            idx = 0
            for ax in reversed(range(dim)):
                idx = idx * dims[ax] + cb[ax]
            cells.append(idx)
            weights.append(w)
    cells = np.asarray(cells, dtype=np.int64)
    weights = np.asarray(weights)
    uc, inv = np.unique(cells, return_inverse=True)
    acc = np.zeros(uc.shape[0])
    np.add.at(acc, inv, weights)
    nz = acc > 0.0
    return uc[nz], acc[nz]


def _trace(p0s, p1s, dims) -> Csr:
    n = int(np.prod(dims))
    rows_c, rows_v = [], []
    for p0, p1 in zip(p0s, p1s):
        c, v = _trace_one(np.asarray(p0, float), np.asarray(p1, float), dims)
        rows_c.append(c)
        rows_v.append(v)
    rowptr = np.zeros(len(rows_c) + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum([c.shape[0] for c in rows_c])
    col = np.concatenate(rows_c).astype(np.int32) if rows_c else np.zeros(0, np.int32)
    val = np.concatenate(rows_v) if rows_v else np.zeros(0)
    return Csr(rowptr, col, val, n)


def trace_rays_2d(nx: int, ny: int, p0s: np.ndarray, p1s: np.ndarray) -> Csr:
    """Straight-ray travel-time operator on an nx x ny grid of [0,1]^2."""
    return _trace(p0s, p1s, (nx, ny))


def trace_rays_3d(nx: int, ny: int, nz: int, p0s: np.ndarray, p1s: np.ndarray) -> Csr:
    """Straight-ray travel-time operator on an nx x ny x nz voxel grid."""
    return _trace(p0s, p1s, (nx, ny, nz))


# ----------------------------------------------------------------------------
# truth and measurements
# ----------------------------------------------------------------------------
def smooth_increment(rng: np.random.Generator, shape, corr_len: float, variance: float):
    """One smooth zero-mean random field on a periodic grid of `shape` (cells
    along each axis of the unit domain), made by convolving white noise with a
    Gaussian of standard deviation `corr_len`; scaled to pointwise `variance`.
    Returned flattened in the cell index order documented above."""
    shape = tuple(int(s) for s in shape)
    white = rng.standard_normal(shape[::-1])  # axis 0 = slowest (last coordinate)
    grids = []
    for ax, n in enumerate(shape[::-1]):
        k = np.arange(n)
        k = np.minimum(k, n - k) / n  # periodic distance in domain units
        grids.append(k)
    mesh = np.meshgrid(*grids, indexing="ij")
    r2 = sum(g * g for g in mesh)
    g = np.exp(-0.5 * r2 / (corr_len * corr_len))
    g /= np.sqrt(np.sum(g * g))
    field = np.real(np.fft.ifftn(np.fft.fftn(white) * np.fft.fftn(g)))
    return (np.sqrt(variance) * field).ravel()


def random_walk_truth(rng, shape, steps: int, corr_len: float, variance: float):
    """s_0 = 0, s_k = s_{k-1} + w_k with smooth increments w_k; shape (steps, N)."""
    n = int(np.prod(shape))
    out = np.zeros((steps, n))
    s = np.zeros(n)
    for k in range(steps):
        s = s + smooth_increment(rng, shape, corr_len, variance)
        out[k] = s
    return out


def _spmv(h: Csr, x: np.ndarray) -> np.ndarray:
    out = np.zeros(h.nrows)
    for i in range(h.nrows):
        a, b = h.rowptr[i], h.rowptr[i + 1]
        out[i] = np.dot(h.val[a:b], x[h.col[a:b]])
    return out


def measurements(rng, h: Csr, truth_k: np.ndarray, noise_var: float):
    """y_k = H s_k + v_k with v_k ~ N(0, noise_var I)."""
    return _spmv(h, truth_k) + np.sqrt(noise_var) * rng.standard_normal(h.nrows)


def tomography_workload(
    grid,
    src,
    rec,
    steps: int,
    corr_len: float,
    variance: float,
    noise_var: float,
    seed: int,
):
    """Fixed-geometry cross-well workload.

    grid: (nx, ny) or (nx, ny, nz); src/rec: counts (2D) or lattice shapes (3D).
    Returns dict(points, H (Csr), truth (steps, N), y (steps, m)).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    if len(grid) == 2:
        nx, ny = grid
        pts = grid_points_2d(nx, ny)
        p0, p1 = cross_well_geometry_2d(int(src), int(rec))
        h = trace_rays_2d(nx, ny, p0, p1)
    else:
        nx, ny, nz = grid
        pts = grid_points_3d(nx, ny, nz)
        p0, p1 = cross_well_geometry_3d(src, rec)
        h = trace_rays_3d(nx, ny, nz, p0, p1)
    truth = random_walk_truth(rng, grid, steps, corr_len, variance)
    y = np.stack([measurements(rng, h, truth[k], noise_var) for k in range(steps)])
    return dict(points=pts, H=h, truth=truth, y=y)


def varying_ray_operators(rng, nx: int, ny: int, ms: Sequence[int]):
    """Time-varying operators: step k uses ms[k] rays between uniformly random
    points of the left and right edges (a new H_k every step)."""
    ops = []
    for m in ms:
        p0 = np.stack([np.zeros(m), rng.uniform(0.02, 0.98, m)], axis=1)
        p1 = np.stack([np.ones(m), rng.uniform(0.02, 0.98, m)], axis=1)
        ops.append(trace_rays_2d(nx, ny, p0, p1))
    return ops
