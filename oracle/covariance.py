"""Exact system-noise covariance Gamma_sys and its products -- test infrastructure.

Gamma(i, j) = kappa(x_i, x_j) with the Matern kernel (Sec. 2.2.1, Eq.
maternfamily).  Three ways to form Gamma X exactly (no hierarchical
compression), all in FP64:

  dense_gamma         -- the full N x N matrix (small N)
  gamma_rows_times    -- rows of Gamma X by direct summation (any N, few rows)
  grid_gamma_times    -- all of Gamma X on a regular grid through the
                         block-Toeplitz structure and the FFT (the alternative
                         the paper names for stationary kernels on equispaced
                         grids, Sec. 2.2.1)
"""

from __future__ import annotations

import numpy as np

from .matern import matern


def pairwise_dist(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    d2 = np.zeros((a.shape[0], b.shape[0]))
    for ax in range(a.shape[1]):
        diff = a[:, ax][:, None] - b[:, ax][None, :]
        d2 += diff * diff
    return np.sqrt(d2)


def dense_gamma(points: np.ndarray, nu: float, ell: float, sigma2: float) -> np.ndarray:
    """The full covariance matrix Gamma_sys (N x N)."""
    return matern(pairwise_dist(points, points), nu, ell, sigma2)


def gamma_rows_times(points, rows, X, nu, ell, sigma2, block=256):
    """(Gamma X)[rows, :] by direct summation over all N points."""
    rows = np.asarray(rows)
    X = np.asarray(X, dtype=np.float64)
    squeeze = X.ndim == 1
    if squeeze:
        X = X[:, None]
    out = np.zeros((rows.shape[0], X.shape[1]))
    for a in range(0, rows.shape[0], block):
        r = rows[a : a + block]
        K = matern(pairwise_dist(points[r], points), nu, ell, sigma2)
        out[a : a + block] = K @ X
    return out[:, 0] if squeeze else out


def gamma_rows_times_sparse_t(points, rows, h, nu, ell, sigma2):
    """(Gamma H^T)[rows, :] for a sparse H (Csr, m x N) by direct summation
    over the nonzeros of H only: G[i, j] = sum_c kappa(x_i, x_c) H[j, c]."""
    rows = np.asarray(rows)
    out = np.zeros((rows.shape[0], h.nrows))
    for j in range(h.nrows):
        a, b = h.rowptr[j], h.rowptr[j + 1]
        cells = h.col[a:b]
        K = matern(pairwise_dist(points[rows], points[cells]), nu, ell, sigma2)
        out[:, j] = K @ h.val[a:b]
    return out


def _grid_symbol(shape, nu, ell, sigma2):
    """FFT of the covariance of a cell-centred grid embedded in a periodic
    grid of twice the size (lag 0..n-1 and -(n-1)..-1; the unused middle lag
    is zero)."""
    lags = []
    for n in shape[::-1]:  # array axis 0 is the slowest coordinate
        k = np.arange(2 * n, dtype=np.float64)
        k = np.where(k < n, k, k - 2 * n)
        lag = k / n
        lag[n] = np.nan
        lags.append(lag)
    mesh = np.meshgrid(*lags, indexing="ij")
    r = np.sqrt(sum(m * m for m in mesh))
    c = matern(np.nan_to_num(r, nan=0.0), nu, ell, sigma2)
    c[np.isnan(r)] = 0.0
    return np.fft.rfftn(c)


def grid_gamma_times(shape, X, nu, ell, sigma2, batch=16, workers=None):
    """Gamma X for the cell centres of a regular grid of `shape` (cells per
    axis on the unit domain; index order: first coordinate fastest).
    workers: threads for the FFTs (scipy.fft), None = numpy's single thread."""
    if workers:
        from scipy import fft as sfft

        rfftn = lambda a, s, axes: sfft.rfftn(a, s=s, axes=axes, workers=workers)  # noqa: E731
        irfftn = lambda a, s, axes: sfft.irfftn(a, s=s, axes=axes, workers=workers)  # noqa: E731
    else:
        rfftn = lambda a, s, axes: np.fft.rfftn(a, s=s, axes=axes)  # noqa: E731
        irfftn = lambda a, s, axes: np.fft.irfftn(a, s=s, axes=axes)  # noqa: E731
    shape = tuple(int(s) for s in shape)
    X = np.asarray(X, dtype=np.float64)
    squeeze = X.ndim == 1
    if squeeze:
        X = X[:, None]
    sym = _grid_symbol(shape, nu, ell, sigma2)
    rshape = shape[::-1]
    pad = tuple(2 * n for n in rshape)
    axes = tuple(range(1, len(rshape) + 1))
    out = np.zeros_like(X)
    for a in range(0, X.shape[1], batch):
        cols = X[:, a : a + batch].T.reshape((-1,) + rshape)
        f = rfftn(cols, pad, axes)
        y = irfftn(f * sym[None], pad, axes)
        sl = (slice(None),) + tuple(slice(0, n) for n in rshape)
        out[:, a : a + batch] = y[sl].reshape(cols.shape[0], -1).T
    return out[:, 0] if squeeze else out
