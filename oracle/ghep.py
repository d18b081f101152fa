"""Generalized Hermitian eigenproblem of the measurement update -- test infrastructure.

The update of one filter step needs the dominant eigenpairs of
    A x = lambda B x,   A = H^T R^-1 H,  B = Gamma^-1            (Eq. ghep)
returned as H^T R^-1 H = Gamma^-1 U Lambda U^T Gamma^-1 with U^T Gamma^-1 U = I
(Eq. geneigendecomposition).  Two ways, both dense FP64 on the CPU:

  ghep_exact       -- the definition: scipy's generalized symmetric eigensolver
                      on (H^T R^-1 H, Gamma^-1), eigenpairs above a relative
                      threshold (the nonzero spectrum);
  ghep_randomized  -- the randomized algorithm of App. B (Alg.
                      randomizedghepuncert), steps in the paper's order:
                      1. Ybar = A Omega for a given Gaussian Omega (N x (k+p));
                      2. QR of Ybar in the B^-1 = Gamma inner product by
                         modified Gram-Schmidt: Qhat^T Gamma Qhat = I;
                      3. Q = B^-1 Qhat = Gamma Qhat, so that Q^T B Q = I;
                      4. T = Q^T A Q (the exact form; the paper also offers an
                         approximation through Omega^T Ybar that saves a second
                         product with A, not needed here);
                      5. T = S Lambda S^T, the k largest modes kept;
                      U = Q S.
"""

from __future__ import annotations

import numpy as np
from scipy import linalg


def ghep_exact(H, R, Gamma, rel_tol=1e-12):
    """Nonzero spectrum of H^T R^-1 H x = lambda Gamma^-1 x: (lam descending, U),
    U^T Gamma^-1 U = I.  Solved as the standard problem of
    Gamma^1/2-conjugation through scipy.linalg.eigh(A, B)."""
    R = np.asarray(R, dtype=np.float64)
    rinv = 1.0 / (np.full(H.shape[0], float(R)) if R.ndim == 0 else R)
    A = H.T @ (rinv[:, None] * H)
    B = np.linalg.inv(Gamma)
    B = 0.5 * (B + B.T)
    lam, V = linalg.eigh(A, B)  # V^T B V = I
    order = np.argsort(lam)[::-1]
    lam, V = lam[order], V[:, order]
    keep = lam > rel_tol * lam[0]
    return lam[keep], V[:, keep]


def mgs_qr_weighted(Y, Wmat):
    """Modified Gram-Schmidt QR of Y in the inner product <x, y> = y^T Wmat x:
    Y = Qh R with Qh^T Wmat Qh = I (Wmat symmetric positive definite)."""
    n, l = Y.shape
    Qh = np.array(Y, dtype=np.float64, copy=True)
    Rm = np.zeros((l, l))
    for j in range(l):
        for i in range(j):
            Rm[i, j] = Qh[:, i] @ (Wmat @ Qh[:, j])
            Qh[:, j] -= Rm[i, j] * Qh[:, i]
        Rm[j, j] = np.sqrt(Qh[:, j] @ (Wmat @ Qh[:, j]))
        Qh[:, j] /= Rm[j, j]
    return Qh, Rm


def ghep_randomized(H, R, Gamma, Omega, k):
    """Alg. randomizedghepuncert for A = H^T R^-1 H, B = Gamma^-1 and the given
    Gaussian Omega (N x (k + p)).  Returns (lam (k, descending), U (N x k)) with
    U^T Gamma^-1 U = I and H^T R^-1 H ~= Gamma^-1 U diag(lam) U^T Gamma^-1."""
    R = np.asarray(R, dtype=np.float64)
    rinv = 1.0 / (np.full(H.shape[0], float(R)) if R.ndim == 0 else R)
    A = H.T @ (rinv[:, None] * H)
    Ybar = A @ Omega                         # step 1
    Qhat, _ = mgs_qr_weighted(Ybar, Gamma)   # step 2: Qhat^T Gamma Qhat = I
    Q = Gamma @ Qhat                         # step 3: Q = B^-1 Qhat, Q^T B Q = I
    T = Q.T @ A @ Q                          # step 4
    T = 0.5 * (T + T.T)
    lam, S = np.linalg.eigh(T)               # step 5
    order = np.argsort(lam)[::-1][:k]
    return lam[order], Q @ S[:, order]
