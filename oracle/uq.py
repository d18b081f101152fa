"""Uncertainty measures from a dense posterior covariance (Sec. 3) -- test infrastructure.

Sigma = Sigma_k|k is an N x N matrix here (from the dense filter); Gamma is the
dense system-noise covariance.  The low-rank pieces the paper works with
(Eq. sigmakk) are recovered densely in `lowrank_from_dense`.

Readings:
  * relative entropy (Sec. 3.2): the paper's log det(alpha I - D) drops the
    (N - r) log alpha term that Sylvester's lemma gives; the quantity computed
    here is H[s|w] = 1/2 (log det Sigma - log det Gamma)
                   = 1/2 (N log alpha + sum_j log(1 - d_j/alpha));
  * realizations (Sec. 3.3): with any factor L_Gamma L_Gamma^T = Gamma and
    X = Gamma^-1 W, the map a = L_Gamma s_u -> s_hat + sqrt(alpha)(a - W Sig X^T a)
    with Sig = I - (I - D/alpha)^(1/2) (the minus root) has covariance Sigma;
    the paper writes alpha_{k+1}^-1 where alpha_k^-1 is meant.
"""

from __future__ import annotations

import numpy as np
from scipy import linalg


def variance(Sigma):
    """Sec. 3.1: the diagonal of Sigma_k|k."""
    return np.diag(Sigma).copy()


def a_optimality_identity(Sigma):
    """Sec. 3.1 with A = I: Trace(Sigma_k|k)."""
    return float(np.trace(Sigma))


def relative_entropy(Sigma, Gamma):
    """Sec. 3.2: H[s_k | w_k] = 1/2 (log det Sigma - log det Gamma)."""
    s1, l1 = np.linalg.slogdet(Sigma)
    s2, l2 = np.linalg.slogdet(Gamma)
    assert s1 > 0 and s2 > 0
    return 0.5 * (l1 - l2)


def lowrank_from_dense(Sigma, Gamma, alpha, rel_tol=1e-12):
    """Recover (W, D) with Sigma = alpha Gamma - W D W^T and W^T Gamma^-1 W = I
    (Eq. sigmakk) from dense matrices: with Gamma = L L^T, the symmetric matrix
    L^-1 (alpha Gamma - Sigma) L^-T = Q diag(d) Q^T gives W = L Q, D = diag(d).
    Eigenvalues below rel_tol * max(|d|) are dropped."""
    L = linalg.cholesky(Gamma, lower=True)
    Mt = linalg.solve_triangular(L, alpha * Gamma - Sigma, lower=True)
    Mt = linalg.solve_triangular(L, Mt.T, lower=True).T
    Mt = 0.5 * (Mt + Mt.T)
    d, Q = np.linalg.eigh(Mt)
    keep = np.abs(d) > rel_tol * max(np.max(np.abs(d)), 1e-300)
    return L @ Q[:, keep], d[keep]


def realization(s_hat, Sigma, Gamma, alpha, a):
    """Conditional realizations s_hat + sqrt(alpha) (a - W Sig X^T a) for the
    columns of a (N x ns), a = L_Gamma s_u (Sec. 3.3, general-factor form)."""
    W, d = lowrank_from_dense(Sigma, Gamma, alpha)
    X = linalg.solve(Gamma, W, assume_a="pos")
    sig = 1.0 - np.sqrt(1.0 - d / alpha)
    a = np.asarray(a, dtype=np.float64)
    return s_hat[:, None] + np.sqrt(alpha) * (a - W @ (sig[:, None] * (X.T @ a)))


def paper_factor(Gamma, W, d, alpha):
    """The factor L = alpha^1/2 (Gamma^1/2 - W Sig W^T Gamma^-1/2) of Sec. 3.3
    with the symmetric square root of Gamma; L L^T = alpha Gamma - W D W^T."""
    ev, V = np.linalg.eigh(Gamma)
    g_half = (V * np.sqrt(ev)) @ V.T
    g_mhalf = (V / np.sqrt(ev)) @ V.T
    sig = 1.0 - np.sqrt(1.0 - d / alpha)
    return np.sqrt(alpha) * (g_half - (W * sig) @ W.T @ g_mhalf)
