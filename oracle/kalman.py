"""Plain Kalman filters with the random-walk forecast -- test infrastructure.

O1 `kf_dense`: Alg. standard (Sec. 2.1, Eqs. prediction, residualcovariance,
kalmangain and the state update) with F_k = I (the random-walk assumption of
Sec. 2.1), written with full N x N matrices.  The covariance update uses the
gain form Sigma+ = Sigma- - K H Sigma-, which equals Eq. filtering
(Sigma- ^-1 + H^T R^-1 H)^-1 by the Woodbury identity and needs no inverse of
Sigma-.  The innovation negative log-likelihood of each step is
    NLL_k = 1/2 (nu^T S^-1 nu + log det S + m log 2 pi),
the Gaussian log-density of the innovation nu = y - H s_pred under N(0, S).

O2 `kf_crosscov_rows`: the same filter for a fixed H, carried in the
cross-covariance variables C = Sigma H^T (N x m), T = H Sigma H^T (m x m) and
c = diag(Sigma).  Every N-indexed quantity is row-local, so the recursion can
be run for any subset of rows; H s is tracked as its own m-vector.  Per step
(Sigma- = Sigma + Gamma):
    C- = C + G, T- = T + A, c- = c + diag(Gamma), S = T- + R,
    z = S^-1 nu, s += C- z, Hs += T- z,
    C = C- - C- S^-1 T-, T = T- - T- S^-1 T-, c = c- - rowsum(C- S^-1 * C-)
with G = Gamma H^T and A = H Gamma H^T.

O1t `kf_dense_truncated`: O1 followed, after every update, by the rank control
of Alg. lowrankaddition step 4 applied to the dense posterior: the correction
alpha_k Gamma - Sigma_k|k is written as W D W^T with W^T Gamma^-1 W = I
(Eq. sigmakk, recovered densely), and only the modes that the low-rank filter
keeps survive: at most r_max of them, the largest merged eigenvalues theta,
and only those with theta > trunc_tol * max(theta).  theta is the eigenvalue
of the merged information term (Sec. 2.4), related to the kept weight by
D = alpha^2 theta / (1 + alpha theta), i.e. theta = d / (alpha (alpha - d)),
which is increasing in d.  The mean update of the next step uses the truncated
covariance, as the low-rank filter does.

O1e `ekf_dense`: the extended Kalman filter of Sec. 4.2 (Alg. extkalman) for the
measurement map y = h(x) + v, h(x) = H s(x), where x is the filtered
(transformed) field and s(x) = ((x + a) / a)^a inverts the Box-Cox transform
x = a (s^(1/a) - 1) of Eq. nonlinear.  Each step linearises h at the predicted
mean: H_k = H diag(s'(x_pred)), s'(x) = ((x + a) / a)^(a - 1); innovation
nu = y - h(x_pred); then the O1 update with H_k (optionally followed by the
truncation of O1t).

Readings (the paper's wording is at odds with itself on these):
  * time index: at step k the filter predicts from k-1 to k and updates with
    y_k (the algorithms use y_k with H s_k);
  * start: s_0 = mu_0 (default 0), Sigma_0|0 = alpha_0 Gamma (default 0, as in
    the experiments of Sec. 4.1.1).
"""

from __future__ import annotations

import numpy as np
from scipy import linalg


def _as_rvec(R, m):
    R = np.asarray(R, dtype=np.float64)
    return np.full(m, float(R)) if R.ndim == 0 else R


def kf_dense(Gamma, steps, s0=None, alpha0=0.0, keep_cov=True):
    """Run O1.  steps: iterable of (y (m,), H (m, N) dense, R scalar or (m,)).

    Returns a list of dicts per step: s (posterior mean), Sigma (posterior
    covariance, if keep_cov), var (its diagonal), nll.
    """
    N = Gamma.shape[0]
    s = np.zeros(N) if s0 is None else np.array(s0, dtype=np.float64)
    Sigma = alpha0 * Gamma.copy()
    out = []
    for y, H, R in steps:
        m = H.shape[0]
        Sigma_p = Sigma + Gamma  # predict with F = I
        nu = y - H @ s
        PHt = Sigma_p @ H.T
        S = H @ PHt + np.diag(_as_rvec(R, m))
        cf = linalg.cho_factor(S, lower=True)
        z = linalg.cho_solve(cf, nu)
        K = linalg.cho_solve(cf, PHt.T).T  # Sigma_p H^T S^-1
        s = s + K @ nu
        Sigma = Sigma_p - K @ PHt.T
        Sigma = 0.5 * (Sigma + Sigma.T)
        logdet = 2.0 * np.sum(np.log(np.diag(cf[0])))
        nll = 0.5 * (nu @ z + logdet + m * np.log(2.0 * np.pi))
        rec = dict(s=s.copy(), var=np.diag(Sigma).copy(), nll=float(nll))
        if keep_cov:
            rec["Sigma"] = Sigma.copy()
        out.append(rec)
    return out


def truncate_lowrank(Sigma, Gamma, alpha, r_max=None, trunc_tol=0.0):
    """Rank control of Alg. lowrankaddition step 4 on a dense posterior.

    alpha Gamma - Sigma = W diag(d) W^T with W^T Gamma^-1 W = I is found densely
    (Gamma = L L^T, L^-1 (alpha Gamma - Sigma) L^-T = Q diag(d) Q^T, W = L Q).
    Modes are ranked by theta = d / (alpha (alpha - d)) (the merged eigenvalue);
    the r_max largest with theta > trunc_tol * max(theta) and theta > 0 are kept.
    Returns (truncated Sigma, kept d (descending), number kept)."""
    L = linalg.cholesky(Gamma, lower=True)
    Mt = linalg.solve_triangular(L, alpha * Gamma - Sigma, lower=True)
    Mt = linalg.solve_triangular(L, Mt.T, lower=True).T
    Mt = 0.5 * (Mt + Mt.T)
    d, Q = np.linalg.eigh(Mt)
    order = np.argsort(d)[::-1]
    d, Q = d[order], Q[:, order]
    theta = np.where(d < alpha, d / (alpha * np.maximum(alpha - d, 1e-300)), np.inf)
    tmax = theta[0] if theta.size else 0.0
    keep = 0
    limit = theta.size if r_max is None else min(r_max, theta.size)
    while keep < limit and theta[keep] > 0 and theta[keep] > trunc_tol * tmax:
        keep += 1
    W = L @ Q[:, :keep]
    Sig = alpha * Gamma - (W * d[:keep]) @ W.T
    return 0.5 * (Sig + Sig.T), d[:keep].copy(), keep


def _kf_update(s, Sigma_p, H, R, y_minus_h):
    m = H.shape[0]
    PHt = Sigma_p @ H.T
    S = H @ PHt + np.diag(_as_rvec(R, m))
    cf = linalg.cho_factor(S, lower=True)
    z = linalg.cho_solve(cf, y_minus_h)
    K = linalg.cho_solve(cf, PHt.T).T
    s = s + K @ y_minus_h
    Sigma = Sigma_p - K @ PHt.T
    Sigma = 0.5 * (Sigma + Sigma.T)
    logdet = 2.0 * np.sum(np.log(np.diag(cf[0])))
    nll = 0.5 * (y_minus_h @ z + logdet + m * np.log(2.0 * np.pi))
    return s, Sigma, float(nll)


def kf_dense_truncated(Gamma, steps, r_max=None, trunc_tol=0.0, s0=None, alpha0=0.0):
    """Run O1t: O1 with the rank control of `truncate_lowrank` after every
    update.  steps: iterable of (y, H dense, R).  Returns per-step dicts with
    s, Sigma, var, nll, r (modes kept) and d (kept weights, descending)."""
    N = Gamma.shape[0]
    s = np.zeros(N) if s0 is None else np.array(s0, dtype=np.float64)
    alpha = alpha0
    Sigma = alpha0 * Gamma.copy()
    out = []
    for y, H, R in steps:
        alpha = alpha + 1.0
        Sigma_p = Sigma + Gamma
        s, Sigma, nll = _kf_update(s, Sigma_p, H, R, y - H @ s)
        Sigma, d, r = truncate_lowrank(Sigma, Gamma, alpha, r_max, trunc_tol)
        out.append(dict(s=s.copy(), Sigma=Sigma.copy(), var=np.diag(Sigma).copy(), nll=nll, r=r, d=d))
    return out


def boxcox_state(x, a):
    """Eq. nonlinear, inverse direction: s = ((x + a) / a)^a."""
    return np.power((np.asarray(x, dtype=np.float64) + a) / a, a)


def boxcox_state_derivative(x, a):
    """ds/dx of `boxcox_state`: ((x + a) / a)^(a - 1)."""
    return np.power((np.asarray(x, dtype=np.float64) + a) / a, a - 1.0)


def ekf_dense(Gamma, steps, a, s0=None, alpha0=0.0, r_max=None, trunc_tol=None):
    """Run O1e (Alg. extkalman written densely).  steps: iterable of
    (y, H dense (m x N), R) with y = H s(x_k) + v.  With r_max / trunc_tol the
    O1t rank control follows every update.  Returns per-step dicts with s (the
    filtered field x), Sigma, var, nll and, when truncating, r and d."""
    N = Gamma.shape[0]
    x = np.zeros(N) if s0 is None else np.array(s0, dtype=np.float64)
    alpha = alpha0
    Sigma = alpha0 * Gamma.copy()
    out = []
    for y, H, R in steps:
        alpha = alpha + 1.0
        Sigma_p = Sigma + Gamma
        Hk = H * boxcox_state_derivative(x, a)[None, :]  # H diag(s'(x_pred))
        nu = y - H @ boxcox_state(x, a)
        x, Sigma, nll = _kf_update(x, Sigma_p, Hk, R, nu)
        rec = dict(nll=nll)
        if r_max is not None or trunc_tol is not None:
            Sigma, d, r = truncate_lowrank(Sigma, Gamma, alpha, r_max, trunc_tol or 0.0)
            rec.update(r=r, d=d)
        rec.update(s=x.copy(), Sigma=Sigma.copy(), var=np.diag(Sigma).copy())
        out.append(rec)
    return out


def kf_dense_randomized_ghep(Gamma, steps, Omega, k, s0=None, alpha0=0.0):
    """The filter of Alg. kalman with the measurement information taken from
    the randomized GHEP of App. B: each step's H^T R^-1 H is replaced by its
    rank-k approximation Gamma^-1 U Lambda U^T Gamma^-1 from
    `ghep.ghep_randomized(H, R, Gamma, Omega, k)` in the covariance update,
    Sigma+ = (Sigma-^-1 + Gamma^-1 U Lambda U^T Gamma^-1)^-1 (written by the
    Woodbury identity, F = Gamma^-1 U:
    Sigma+ = Sigma- - Sigma- F (Lambda^-1 + F^T Sigma- F)^-1 F^T Sigma-),
    while the mean, the innovation covariance and the NLL use the exact
    Kalman update with Sigma- (Alg. kalman computes the gain from
    Sigma H^T directly).  Returns per-step dicts with s, Sigma, var, nll."""
    from . import ghep

    N = Gamma.shape[0]
    s = np.zeros(N) if s0 is None else np.array(s0, dtype=np.float64)
    Sigma = alpha0 * Gamma.copy()
    out = []
    for y, H, R in steps:
        Sigma_p = Sigma + Gamma
        s, _, nll = _kf_update(s, Sigma_p, H, R, y - H @ s)
        lam, U = ghep.ghep_randomized(H, R, Gamma, Omega, k)
        F = np.linalg.solve(Gamma, U)
        SF = Sigma_p @ F
        inner = np.diag(1.0 / lam) + F.T @ SF
        Sigma = Sigma_p - SF @ np.linalg.solve(inner, SF.T)
        Sigma = 0.5 * (Sigma + Sigma.T)
        out.append(dict(s=s.copy(), Sigma=Sigma.copy(), var=np.diag(Sigma).copy(), nll=nll))
    return out


def kf_information_form(Gamma, steps, alpha0=0.0):
    """Covariances only, via Eq. filtering: Sigma+ = (Sigma-^-1 + H^T R^-1 H)^-1.
    Used to pin O1 by a second, independent algebra (requires Sigma- SPD, i.e.
    alpha0 + k > 0)."""
    Sigma = alpha0 * Gamma.copy()
    out = []
    for _, H, R in steps:
        m = H.shape[0]
        Sigma_p = Sigma + Gamma
        info = np.linalg.inv(Sigma_p) + H.T @ np.diag(1.0 / _as_rvec(R, m)) @ H
        Sigma = np.linalg.inv(info)
        Sigma = 0.5 * (Sigma + Sigma.T)
        out.append(Sigma.copy())
    return out


def kf_crosscov_rows(G_rows, A, diag_gamma_rows, HG_full_rows_y, alpha0=0.0):
    """Run O2 on a subset of rows for a fixed H.

    G_rows: (n_rows, m) rows of G = Gamma H^T; A: (m, m) = H Gamma H^T;
    diag_gamma_rows: (n_rows,) diag(Gamma) on those rows;
    HG_full_rows_y: iterable of (y (m,), R scalar or (m,)).
    Start: s_0 = 0 and Sigma_0 = alpha0 Gamma.
    Returns per-step dicts: s_rows, var_rows, nll.
    """
    n, m = G_rows.shape
    C = alpha0 * G_rows.copy()
    T = alpha0 * A.copy()
    c = alpha0 * np.array(diag_gamma_rows, dtype=np.float64)
    s = np.zeros(n)
    hs = np.zeros(m)
    out = []
    for y, R in HG_full_rows_y:
        Cp = C + G_rows
        Tp = T + A
        cp = c + diag_gamma_rows
        S = Tp + np.diag(_as_rvec(R, m))
        cf = linalg.cho_factor(S, lower=True)
        nu = y - hs
        z = linalg.cho_solve(cf, nu)
        s = s + Cp @ z
        hs = hs + Tp @ z
        SiT = linalg.cho_solve(cf, Tp)
        SiCt = linalg.cho_solve(cf, Cp.T)
        C = Cp - Cp @ SiT
        T = Tp - Tp @ SiT
        T = 0.5 * (T + T.T)
        c = cp - np.einsum("ij,ji->i", Cp, SiCt)
        logdet = 2.0 * np.sum(np.log(np.diag(cf[0])))
        nll = 0.5 * (nu @ z + logdet + m * np.log(2.0 * np.pi))
        out.append(dict(s_rows=s.copy(), var_rows=c.copy(), nll=float(nll)))
    return out


def scalar_closed_form(gamma, h, rho, steps, alpha0=0.0):
    """N = m = 1 random walk: Sigma_k = e_k gamma with e = alpha - d; the
    predict adds 1 to e, the update maps e -> 1/(1/e + lam) with
    lam = h^2 gamma / rho (the per-mode form of the D recurrence of
    Alg. kalmanconstantH).  Returns the list of Sigma_k."""
    lam = h * h * gamma / rho
    e = alpha0
    out = []
    for _ in range(steps):
        e = e + 1.0
        e = 1.0 / (1.0 / e + lam)
        out.append(e * gamma)
    return out


def scalar_steady_state(gamma, h, rho):
    """Fixed point of the scalar recurrence: e = 1/(1/(e+1) + lam), i.e.
    lam e^2 + lam e - 1 = 0 -> e = (-lam + sqrt(lam^2 + 4 lam)) / (2 lam)."""
    lam = h * h * gamma / rho
    return gamma * (-lam + np.sqrt(lam * lam + 4.0 * lam)) / (2.0 * lam)


def nll_batch_and_gradients(Gamma1, sigma2, rho, Hs, ys, s0=None, alpha0=0.0):
    """The summed innovation NLL of K filter steps and its exact gradients, from
    the joint Gaussian of all measurements (prediction-error decomposition):

        Y ~ N(mu, C),  mu_k = H_k s0,
        C[i, j] = (alpha0 + min(i, j)) sigma2 H_i Gamma1 H_j^T + delta_ij rho I
        (steps i, j counted from 1; s_k = s0 + w_1 + ... + w_k, Gamma = sigma2 Gamma1),
        NLL = 1/2 (Y - mu)^T C^-1 (Y - mu) + 1/2 log det C + M/2 log 2 pi.

    Gradients: dNLL/dY = C^-1 (Y - mu) =: q; dNLL/ds0 = -sum_k H_k^T q_k;
    dNLL/dtheta = 1/2 tr(C^-1 dC) - 1/2 q^T dC q for theta in {sigma2, rho}
    (dC/dsigma2 = C_Gamma / sigma2, dC/drho = I).
    Returns (nll, grad_y (list of m_k arrays), grad_s0, grad_sigma2, grad_rho)."""
    K = len(Hs)
    N = Gamma1.shape[0]
    s0 = np.zeros(N) if s0 is None else np.asarray(s0, dtype=np.float64)
    ms = [H.shape[0] for H in Hs]
    off = np.concatenate([[0], np.cumsum(ms)]).astype(int)
    M = int(off[-1])
    CG = np.zeros((M, M))
    for i in range(K):
        for j in range(K):
            CG[off[i] : off[i + 1], off[j] : off[j + 1]] = (alpha0 + min(i, j) + 1) * sigma2 * (
                Hs[i] @ Gamma1 @ Hs[j].T)
    C = CG + rho * np.eye(M)
    Y = np.concatenate([np.asarray(y, dtype=np.float64) for y in ys])
    mu = np.concatenate([H @ s0 for H in Hs])
    cf = linalg.cho_factor(C, lower=True)
    d = Y - mu
    q = linalg.cho_solve(cf, d)
    logdet = 2.0 * np.sum(np.log(np.diag(cf[0])))
    nll = 0.5 * (d @ q + logdet + M * np.log(2.0 * np.pi))
    Ci = linalg.cho_solve(cf, np.eye(M))
    g_sigma2 = 0.5 * (np.sum(Ci * CG) - q @ CG @ q) / sigma2
    g_rho = 0.5 * (np.trace(Ci) - q @ q)
    g_y = [q[off[k] : off[k + 1]].copy() for k in range(K)]
    g_s0 = -sum(Hs[k].T @ g_y[k] for k in range(K))
    return float(nll), g_y, g_s0, float(g_sigma2), float(g_rho)
