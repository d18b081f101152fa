"""Matern covariance kernel (Sec. 2.2.1, Eq. maternfamily) -- test infrastructure.

The paper writes C(r) = (sqrt(2 nu) a r)^nu K_nu(sqrt(2 nu) a r) / (2^(nu-1) Gamma(nu))
with an inverse length scale a and no variance factor.  Reading used here: a =
1/ell and an explicit variance sigma2 multiplies the kernel, so C(0) = sigma2.
For nu = 1/2 + n the kernel is an exponential times a polynomial of order n
(stated below the equation); the two closed forms used by the workloads are

    nu = 1/2 :  sigma2 * exp(-r/ell)
    nu = 3/2 :  sigma2 * (1 + sqrt(3) r/ell) * exp(-sqrt(3) r/ell)
"""

from __future__ import annotations

import numpy as np
from scipy import special


def matern_general(r, nu: float, ell: float, sigma2: float = 1.0):
    """Eq. maternfamily written out with the Bessel function K_nu (r > 0)."""
    r = np.asarray(r, dtype=np.float64)
    z = np.sqrt(2.0 * nu) * r / ell
    out = np.empty_like(z)
    zero = z == 0.0
    zz = z[~zero]
    out[~zero] = sigma2 * (zz**nu) * special.kv(nu, zz) / (2.0 ** (nu - 1.0) * special.gamma(nu))
    out[zero] = sigma2
    return out


def matern(r, nu: float, ell: float, sigma2: float = 1.0):
    """Closed forms for nu in {1/2, 3/2}; any other nu uses matern_general."""
    r = np.asarray(r, dtype=np.float64)
    if nu == 0.5:
        return sigma2 * np.exp(-r / ell)
    if nu == 1.5:
        z = np.sqrt(3.0) * r / ell
        return sigma2 * (1.0 + z) * np.exp(-z)
    return matern_general(r, nu, ell, sigma2)
