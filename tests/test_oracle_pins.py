"""Pins for the CPU oracle and the input generators (no GPU).

Each test checks the oracle against something other than itself: a closed
form, a library routine, a second independent algebra, or brute force.
"""

import numpy as np
import pytest
from scipy import linalg, special, stats

from oracle import covariance, ghep, kalman, matern, uq
import synth


# ----------------------------------------------------------------------------
# Matern kernel (Sec. 2.2.1, Eq. maternfamily)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("nu", [0.5, 1.5])
def test_matern_closed_forms_match_bessel_formula(nu):
    """The nu = 1/2 and 3/2 closed forms equal the K_nu formula (scipy kv)."""
    r = np.linspace(1e-4, 3.0, 400)
    for ell in (0.05, 0.2, 1.0):
        a = matern.matern(r, nu, ell, 2.5)
        b = matern.matern_general(r, nu, ell, 2.5)
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-300)


def test_matern_general_nu_5_2_textbook_form():
    """nu = 5/2: sigma2 (1 + z + z^2/3) e^-z with z = sqrt(5) r / ell; also
    C(0) = sigma2 (continuity at r = 0)."""
    r = np.linspace(1e-6, 2.0, 100)
    z = np.sqrt(5.0) * r / 0.3
    ref = 1.7 * (1 + z + z * z / 3) * np.exp(-z)
    np.testing.assert_allclose(matern.matern_general(r, 2.5, 0.3, 1.7), ref, rtol=1e-11)
    assert matern.matern_general(np.array([0.0]), 2.5, 0.3, 1.7)[0] == 1.7
    assert abs(matern.matern_general(np.array([1e-9]), 1.5, 0.3, 1.7)[0] - 1.7) < 1e-7


# ----------------------------------------------------------------------------
# ray tracer (Eq. lineartomography)
# ----------------------------------------------------------------------------
def test_ray_row_sums_equal_ray_lengths():
    p0, p1 = synth.cross_well_geometry_2d(8, 4)
    h = synth.trace_rays_2d(32, 32, p0, p1)
    lengths = np.hypot(p1[:, 0] - p0[:, 0], p1[:, 1] - p0[:, 1])
    sums = np.add.reduceat(h.val, h.rowptr[:-1])
    np.testing.assert_allclose(sums, lengths, rtol=1e-14)
    assert np.all(h.val > 0)
    # columns sorted and unique within each row
    for i in range(h.nrows):
        c = h.col[h.rowptr[i] : h.rowptr[i + 1]]
        assert np.all(np.diff(c) > 0)


def test_ray_through_cell_centres_and_along_grid_line():
    # horizontal ray through a row of cell centres: length 1/nx in each cell
    h = synth.trace_rays_2d(4, 4, np.array([[0, 0.375]]), np.array([[1, 0.375]]))
    np.testing.assert_array_equal(h.col, [4, 5, 6, 7])
    np.testing.assert_allclose(h.val, 0.25)
    # a ray along the grid line y = 1/2 is shared equally by the two rows
    h = synth.trace_rays_2d(4, 4, np.array([[0, 0.5]]), np.array([[1, 0.5]]))
    np.testing.assert_array_equal(h.col, [4, 5, 6, 7, 8, 9, 10, 11])
    np.testing.assert_allclose(h.val, 0.125)
    # diagonal of the square through grid vertices: sqrt(2)/n in each diagonal cell
    h = synth.trace_rays_2d(5, 5, np.array([[0, 0.0]]), np.array([[1, 1.0]]))
    np.testing.assert_array_equal(h.col, [0, 6, 12, 18, 24])
    np.testing.assert_allclose(h.val, np.sqrt(2) / 5)


def test_ray_3d_row_sums():
    p0, p1 = synth.cross_well_geometry_3d((2, 3), (3, 2))
    h = synth.trace_rays_3d(6, 5, 4, p0, p1)
    lengths = np.linalg.norm(p1 - p0, axis=1)
    sums = np.add.reduceat(h.val, h.rowptr[:-1])
    np.testing.assert_allclose(sums, lengths, rtol=1e-13)


# ----------------------------------------------------------------------------
# exact Gamma products
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(7, 5), (4, 3, 5), (16, 16)])
def test_grid_fft_product_equals_dense(shape):
    rng = np.random.default_rng(1)
    pts = synth.grid_points_2d(*shape) if len(shape) == 2 else synth.grid_points_3d(*shape)
    G = covariance.dense_gamma(pts, 1.5, 0.3, 1.3)
    X = rng.standard_normal((pts.shape[0], 5))
    for workers in (None, 2):
        Y = covariance.grid_gamma_times(shape, X, 1.5, 0.3, 1.3, workers=workers)
        np.testing.assert_allclose(Y, G @ X, rtol=0, atol=1e-12 * np.abs(G @ X).max())


def test_direct_row_sums_equal_dense():
    rng = np.random.default_rng(2)
    pts = rng.uniform(size=(300, 2))
    G = covariance.dense_gamma(pts, 0.5, 0.1, 1.0)
    X = rng.standard_normal((300, 3))
    rows = np.array([0, 17, 299])
    np.testing.assert_allclose(covariance.gamma_rows_times(pts, rows, X, 0.5, 0.1, 1.0), (G @ X)[rows], rtol=1e-13)
    p0, p1 = synth.cross_well_geometry_2d(3, 3)
    pts = synth.grid_points_2d(10, 10)
    h = synth.trace_rays_2d(10, 10, p0, p1)
    G = covariance.dense_gamma(pts, 0.5, 0.1, 1.0)
    Hd = synth.csr_to_dense(h)
    rows = np.arange(0, 100, 7)
    np.testing.assert_allclose(covariance.gamma_rows_times_sparse_t(pts, rows, h, 0.5, 0.1, 1.0), (G @ Hd.T)[rows], rtol=1e-13)


# ----------------------------------------------------------------------------
# O1: dense Kalman filter
# ----------------------------------------------------------------------------
def test_kf_dense_scalar_closed_form_and_steady_state():
    """N = m = 1: Sigma_k follows e <- 1/(1/(e+1) + lam) and converges to the
    root of lam e^2 + lam e - 1 = 0."""
    gamma, h, rho = 0.7, 1.3, 0.05
    steps = [(np.array([0.1 * k]), np.array([[h]]), rho) for k in range(200)]
    res = kalman.kf_dense(np.array([[gamma]]), steps)
    ref = kalman.scalar_closed_form(gamma, h, rho, 200)
    np.testing.assert_allclose([r["Sigma"][0, 0] for r in res], ref, rtol=1e-13)
    assert abs(res[-1]["Sigma"][0, 0] - kalman.scalar_steady_state(gamma, h, rho)) < 1e-14


def _random_problem(rng, N, ms, alpha0=0.0):
    pts = rng.uniform(size=(N, 2))
    Gamma = covariance.dense_gamma(pts, 1.5, 0.3, 1.0)
    steps = []
    for m in ms:
        H = rng.standard_normal((m, N))
        steps.append((rng.standard_normal(m), H, rng.uniform(0.05, 0.2, m)))
    return Gamma, steps


def test_kf_dense_matches_information_form():
    """Gain form (O1) == Eq. filtering (inverse of Sigma-^-1 + H^T R^-1 H)."""
    rng = np.random.default_rng(3)
    Gamma, steps = _random_problem(rng, 12, [3, 5, 2, 4, 6])
    a = kalman.kf_dense(Gamma, steps, alpha0=0.5)
    b = kalman.kf_information_form(Gamma, steps, alpha0=0.5)
    for ra, Sb in zip(a, b):
        np.testing.assert_allclose(ra["Sigma"], Sb, rtol=1e-10, atol=1e-12)


def _batch_gaussian(Gamma, steps, alpha0):
    """Joint Gaussian of (s_K, y_1..y_K) under s_k = s_0 + w_1 + ... + w_k:
    Cov(s_i, s_j) = (alpha0 + min(i, j)) Gamma."""
    K = len(steps)
    Hs = [H for _, H, _ in steps]
    ms = [H.shape[0] for H in Hs]
    off = np.concatenate([[0], np.cumsum(ms)])
    Cyy = np.zeros((off[-1], off[-1]))
    Csy = np.zeros((Gamma.shape[0], off[-1]))
    for i in range(K):
        for j in range(K):
            Cyy[off[i] : off[i + 1], off[j] : off[j + 1]] = (alpha0 + min(i, j) + 1) * Hs[i] @ Gamma @ Hs[j].T
        R = np.asarray(steps[i][2], dtype=float)
        Cyy[off[i] : off[i + 1], off[i] : off[i + 1]] += np.diag(np.broadcast_to(R, (ms[i],)))
        Csy[:, off[i] : off[i + 1]] = (alpha0 + min(K - 1, i) + 1) * Gamma @ Hs[i].T
    Y = np.concatenate([y for y, _, _ in steps])
    return Cyy, Csy, Y


def test_kf_dense_equals_batch_posterior_and_likelihood():
    """After K steps the filter's mean/covariance equal the batch Gaussian
    conditional of s_K given all y, and the summed innovation NLL equals
    -log N(Y; 0, Cov(Y)) (prediction-error decomposition)."""
    rng = np.random.default_rng(4)
    Gamma, steps = _random_problem(rng, 9, [2, 4, 3, 3])
    alpha0 = 0.3
    res = kalman.kf_dense(Gamma, steps, alpha0=alpha0)
    Cyy, Csy, Y = _batch_gaussian(Gamma, steps, alpha0)
    s_batch = Csy @ np.linalg.solve(Cyy, Y)
    Sig_batch = (alpha0 + len(steps)) * Gamma - Csy @ np.linalg.solve(Cyy, Csy.T)
    np.testing.assert_allclose(res[-1]["s"], s_batch, rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(res[-1]["Sigma"], Sig_batch, rtol=1e-9, atol=1e-11)
    nll_batch = -stats.multivariate_normal(mean=np.zeros(Y.shape[0]), cov=Cyy).logpdf(Y)
    assert abs(sum(r["nll"] for r in res) - nll_batch) < 1e-9 * abs(nll_batch)


# ----------------------------------------------------------------------------
# O2: cross-covariance recursion on sampled rows
# ----------------------------------------------------------------------------
def test_crosscov_rows_match_dense_filter():
    rng = np.random.default_rng(5)
    N, m = 40, 6
    Gamma, _ = _random_problem(rng, N, [])
    H = rng.standard_normal((m, N))
    ys = [(rng.standard_normal(m), 0.1) for _ in range(7)]
    dense = kalman.kf_dense(Gamma, [(y, H, R) for y, R in ys], alpha0=0.2)
    rows = np.array([0, 5, 11, 39])
    G = Gamma @ H.T
    o2 = kalman.kf_crosscov_rows(G[rows], H @ G, np.diag(Gamma)[rows], ys, alpha0=0.2)
    for a, b in zip(dense, o2):
        np.testing.assert_allclose(b["s_rows"], a["s"][rows], rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(b["var_rows"], a["var"][rows], rtol=1e-10, atol=1e-12)
        assert abs(a["nll"] - b["nll"]) < 1e-10 * max(1.0, abs(a["nll"]))


# ----------------------------------------------------------------------------
# Sec. 3 uncertainty measures
# ----------------------------------------------------------------------------
def test_lowrank_factor_realization_and_entropy():
    rng = np.random.default_rng(6)
    Gamma, steps = _random_problem(rng, 15, [3, 3, 4])
    res = kalman.kf_dense(Gamma, steps)
    Sigma = res[-1]["Sigma"]
    alpha = float(len(steps))
    W, d = uq.lowrank_from_dense(Sigma, Gamma, alpha)
    # Eq. sigmakk and the Gamma^-1-orthonormality of W
    np.testing.assert_allclose(alpha * Gamma - (W * d) @ W.T, Sigma, atol=1e-10)
    np.testing.assert_allclose(W.T @ np.linalg.solve(Gamma, W), np.eye(W.shape[1]), atol=1e-9)
    assert np.all(d > 0) and np.all(d < alpha) and W.shape[1] <= 10
    # the Sec. 3.3 factor with the symmetric square root: L L^T = Sigma
    L = uq.paper_factor(Gamma, W, d, alpha)
    np.testing.assert_allclose(L @ L.T, Sigma, atol=1e-9)
    # the general-factor map a = chol(Gamma) s_u: its linear part has L' L'^T = Sigma
    Lg = linalg.cholesky(Gamma, lower=True)
    x = uq.realization(np.zeros(15), Sigma, Gamma, alpha, Lg)
    np.testing.assert_allclose(x @ x.T, Sigma, atol=1e-9)
    # relative entropy via Sylvester: 1/2 (N log alpha + sum log(1 - d/alpha))
    ent = 0.5 * (15 * np.log(alpha) + np.sum(np.log(1.0 - d / alpha)))
    assert abs(uq.relative_entropy(Sigma, Gamma) - ent) < 1e-8
    assert abs(uq.a_optimality_identity(Sigma) - (alpha * np.trace(Gamma) - np.sum(d * np.sum(W * W, axis=0)))) < 1e-9


def test_generator_is_deterministic_and_shaped():
    a = synth.tomography_workload((16, 12), 4, 3, 3, 0.1, 1.0, 1e-4, seed=synth.BASE_SEED)
    b = synth.tomography_workload((16, 12), 4, 3, 3, 0.1, 1.0, 1e-4, seed=synth.BASE_SEED)
    np.testing.assert_array_equal(a["y"], b["y"])
    assert a["truth"].shape == (3, 192) and a["y"].shape == (3, 12)
    inc = np.diff(np.vstack([np.zeros(192), a["truth"]]), axis=0)
    assert 0.3 < inc.var() < 3.0


def test_batch_gradients_match_central_differences_of_dense_kf():
    """The batch-Gaussian gradients are pinned by central finite differences of
    the dense filter's summed NLL (a different algebra: the recursion)."""
    rng = np.random.default_rng(8)
    N, ms = 10, [3, 4, 3]
    pts = rng.uniform(size=(N, 2))
    G1 = covariance.dense_gamma(pts, 1.5, 0.3, 1.0)
    Hs = [rng.standard_normal((m, N)) for m in ms]
    ys = [rng.standard_normal(m) for m in ms]
    s0 = rng.standard_normal(N)
    sigma2, rho, alpha0 = 0.7, 0.05, 0.4

    def total(sig, r, yv, s):
        res = kalman.kf_dense(sig * G1, [(yv[k], Hs[k], r) for k in range(len(ms))], s0=s, alpha0=alpha0,
                              keep_cov=False)
        return sum(x["nll"] for x in res)

    nll, gy, gs0, gsig, grho = kalman.nll_batch_and_gradients(G1, sigma2, rho, Hs, ys, s0, alpha0)
    assert abs(nll - total(sigma2, rho, ys, s0)) < 1e-10 * abs(nll)
    h = 1e-6
    fd_sig = (total(sigma2 + h, rho, ys, s0) - total(sigma2 - h, rho, ys, s0)) / (2 * h)
    fd_rho = (total(sigma2, rho + h, ys, s0) - total(sigma2, rho - h, ys, s0)) / (2 * h)
    assert abs(fd_sig - gsig) < 1e-6 * max(1, abs(gsig))
    assert abs(fd_rho - grho) < 1e-6 * max(1, abs(grho))
    for k, j in [(0, 1), (2, 2), (1, 0)]:
        yp = [y.copy() for y in ys]
        ym = [y.copy() for y in ys]
        yp[k][j] += h
        ym[k][j] -= h
        fd = (total(sigma2, rho, yp, s0) - total(sigma2, rho, ym, s0)) / (2 * h)
        assert abs(fd - gy[k][j]) < 1e-6 * max(1, abs(fd))
    for i in (0, 7):
        sp, sm_ = s0.copy(), s0.copy()
        sp[i] += h
        sm_[i] -= h
        fd = (total(sigma2, rho, ys, sp) - total(sigma2, rho, ys, sm_)) / (2 * h)
        assert abs(fd - gs0[i]) < 1e-6 * max(1, abs(fd))


# ----------------------------------------------------------------------------
# O1t: rank control of the low-rank posterior (Alg. lowrankaddition step 4)
# ----------------------------------------------------------------------------
def test_truncation_equals_generalized_eigen_truncation():
    """truncate_lowrank keeps the leading generalized eigenpairs of
    (alpha Gamma - Sigma) u = d Gamma u (scipy's generalized eigensolver, an
    independent route), and the whitened error equals the first dropped d
    (best rank-r approximation in the Gamma^-1 metric)."""
    rng = np.random.default_rng(21)
    Gamma, steps = _random_problem(rng, 25, [4, 5, 3])
    res = kalman.kf_dense(Gamma, steps)
    alpha = float(len(steps))
    Sigma = res[-1]["Sigma"]
    Delta = alpha * Gamma - Sigma
    d_all, U = linalg.eigh(0.5 * (Delta + Delta.T), Gamma)  # U^T Gamma U = I
    d_all, U = d_all[::-1], U[:, ::-1]
    for r_max in (3, 7, 11):
        St, d, r = kalman.truncate_lowrank(Sigma, Gamma, alpha, r_max=r_max)
        assert r == r_max
        np.testing.assert_allclose(d, d_all[:r_max], rtol=1e-9, atol=1e-12)
        W = Gamma @ U[:, :r_max]
        ref = alpha * Gamma - (W * d_all[:r_max]) @ W.T
        np.testing.assert_allclose(St, ref, rtol=1e-9, atol=1e-11)
        L = np.linalg.cholesky(Gamma)
        E = linalg.solve_triangular(L, St - Sigma, lower=True)
        E = linalg.solve_triangular(L, E.T, lower=True).T
        assert abs(np.linalg.norm(E, 2) - d_all[r_max]) < 1e-8 * d_all[0]
    # rank of the correction after 3 steps is at most sum m_k = 12
    assert np.sum(d_all > 1e-10 * d_all[0]) <= 12


def test_truncated_filter_without_cap_is_o1_and_caps_rank():
    rng = np.random.default_rng(22)
    Gamma, steps = _random_problem(rng, 20, [3, 4, 2, 5])
    a = kalman.kf_dense(Gamma, steps)
    b = kalman.kf_dense_truncated(Gamma, steps, r_max=None, trunc_tol=0.0)
    for x, y in zip(a, b):
        np.testing.assert_allclose(y["Sigma"], x["Sigma"], rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(y["s"], x["s"], rtol=1e-10, atol=1e-12)
        assert abs(x["nll"] - y["nll"]) < 1e-10 * abs(x["nll"])
    c = kalman.kf_dense_truncated(Gamma, steps, r_max=5, trunc_tol=1e-12)
    assert [q["r"] for q in c] == [3, 5, 5, 5]
    # every truncated posterior stays symmetric positive definite
    for q in c:
        assert np.linalg.eigvalsh(q["Sigma"]).min() > 0
    # trunc_tol: theta = d / (alpha (alpha - d)) of every kept mode above tol * max
    e = kalman.kf_dense_truncated(Gamma, steps, trunc_tol=1e-2)
    for k, q in enumerate(e):
        al = k + 1.0
        th = q["d"] / (al * (al - q["d"]))
        assert np.all(th > 1e-2 * th[0])


# ----------------------------------------------------------------------------
# O1e: extended Kalman filter with the Box-Cox map (Sec. 4.2, Alg. extkalman)
# ----------------------------------------------------------------------------
def test_boxcox_map_inverse_derivative_and_log_limit():
    """s(x) inverts Eq. nonlinear's x = a (s^(1/a) - 1); its derivative matches
    central differences; a -> infinity gives s = exp(x) (the log-transform
    limit the paper names)."""
    x = np.linspace(-0.9, 2.0, 37)
    for a in (1.0, 2.0, 4.0, 6.0, 2.5):
        s = kalman.boxcox_state(x, a)
        np.testing.assert_allclose(a * (s ** (1.0 / a) - 1.0), x, rtol=1e-12, atol=1e-13)
        h = 1e-6
        fd = (kalman.boxcox_state(x + h, a) - kalman.boxcox_state(x - h, a)) / (2 * h)
        np.testing.assert_allclose(kalman.boxcox_state_derivative(x, a), fd, rtol=1e-7)
    np.testing.assert_allclose(kalman.boxcox_state(x, 1e8), np.exp(x), rtol=1e-6)


def test_ekf_with_identity_map_is_the_linear_filter():
    """a = 1: s(x) = x + 1 is affine with unit Jacobian, so the EKF equals O1
    on the measurements y - H 1."""
    rng = np.random.default_rng(23)
    Gamma, steps = _random_problem(rng, 15, [3, 4, 2])
    a = kalman.ekf_dense(Gamma, steps, 1.0)
    b = kalman.kf_dense(Gamma, [(y - H @ np.ones(15), H, R) for y, H, R in steps])
    for x, y in zip(a, b):
        np.testing.assert_allclose(x["s"], y["s"], rtol=1e-11, atol=1e-12)
        np.testing.assert_allclose(x["Sigma"], y["Sigma"], rtol=1e-11, atol=1e-12)
        assert abs(x["nll"] - y["nll"]) < 1e-11 * abs(y["nll"])


def test_ekf_step_is_one_gauss_newton_step():
    """One EKF step from (x0, Sigma-) equals one Gauss-Newton step of the MAP
    objective 1/2 |y - h(x)|^2_R^-1 + 1/2 |x - x0|^2_Sigma-^-1 started at x0,
    solved as a stacked whitened least-squares problem (numpy lstsq)."""
    rng = np.random.default_rng(24)
    N, m, a = 18, 5, 4.0
    Gamma, _ = _random_problem(rng, N, [])
    H = np.abs(rng.standard_normal((m, N)))
    R = rng.uniform(0.05, 0.2, m)
    x0 = 0.3 * rng.standard_normal(N)
    Sig0 = 0.5 * Gamma
    y = H @ kalman.boxcox_state(x0 + 0.1 * rng.standard_normal(N), a)
    out = kalman.ekf_dense(Gamma, [(y, H, R)], a, s0=x0, alpha0=0.5)
    J = H * kalman.boxcox_state_derivative(x0, a)[None, :]
    Lp = np.linalg.cholesky(Sig0 + Gamma)
    top = J / np.sqrt(R)[:, None]
    bot = linalg.solve_triangular(Lp, np.eye(N), lower=True)
    rhs = np.concatenate([(y - H @ kalman.boxcox_state(x0, a)) / np.sqrt(R), np.zeros(N)])
    delta = np.linalg.lstsq(np.vstack([top, bot]), rhs, rcond=None)[0]
    np.testing.assert_allclose(out[0]["s"], x0 + delta, rtol=1e-9, atol=1e-11)


# ----------------------------------------------------------------------------
# Eq. ghep: exact and randomized (App. B, Alg. randomizedghepuncert)
# ----------------------------------------------------------------------------
def _ghep_problem(rng, N=40, m=9):
    pts = rng.uniform(size=(N, 2))
    Gamma = covariance.dense_gamma(pts, 1.5, 0.3, 1.0)
    H = rng.standard_normal((m, N))
    R = rng.uniform(0.05, 0.2, m)
    return Gamma, H, R


def test_ghep_exact_identities_and_data_space_spectrum():
    """U^T Gamma^-1 U = I, Gamma^-1 U Lambda U^T Gamma^-1 = H^T R^-1 H
    (Eq. geneigendecomposition), and the nonzero eigenvalues are those of the
    data-space matrix R^-1/2 H Gamma H^T R^-1/2 (numpy eigvalsh)."""
    rng = np.random.default_rng(31)
    Gamma, H, R = _ghep_problem(rng)
    lam, U = ghep.ghep_exact(H, R, Gamma)
    assert lam.shape[0] == H.shape[0]
    Gi = np.linalg.inv(Gamma)
    np.testing.assert_allclose(U.T @ Gi @ U, np.eye(lam.shape[0]), atol=1e-9)
    A = H.T @ (H / R[:, None])
    np.testing.assert_allclose(Gi @ (U * lam) @ U.T @ Gi, A, rtol=0, atol=1e-8 * np.abs(A).max())
    rs = 1.0 / np.sqrt(R)
    ds = np.linalg.eigvalsh((rs[:, None] * (H @ Gamma @ H.T)) * rs[None, :])[::-1]
    np.testing.assert_allclose(lam, ds, rtol=1e-9)


def test_mgs_qr_in_weighted_inner_product():
    rng = np.random.default_rng(32)
    Gamma, _, _ = _ghep_problem(rng)
    Y = rng.standard_normal((Gamma.shape[0], 7))
    Qh, Rm = ghep.mgs_qr_weighted(Y, Gamma)
    np.testing.assert_allclose(Qh.T @ Gamma @ Qh, np.eye(7), atol=1e-12)
    np.testing.assert_allclose(Qh @ Rm, Y, rtol=1e-12, atol=1e-12)
    assert np.allclose(np.tril(Rm, -1), 0)


def test_randomized_ghep_exact_when_sketch_spans_range():
    """k + p = rank(A): the sketch spans the range of B^-1 A, so the randomized
    algorithm returns the exact nonzero spectrum; also for an A of exact rank
    k < m (a rank-deficient H).  (A sketch wider than the rank would ask the
    Gram-Schmidt step to normalise rounding noise.)"""
    rng = np.random.default_rng(33)
    Gamma, H, R = _ghep_problem(rng)
    lam, U = ghep.ghep_exact(H, R, Gamma)
    Om = rng.standard_normal((Gamma.shape[0], H.shape[0]))
    lr, Ur = ghep.ghep_randomized(H, R, Gamma, Om, H.shape[0])
    np.testing.assert_allclose(lr, lam, rtol=1e-9)
    Gi = np.linalg.inv(Gamma)
    A = H.T @ (H / R[:, None])
    np.testing.assert_allclose(Gi @ (Ur * lr) @ Ur.T @ Gi, A, rtol=0, atol=1e-8 * np.abs(A).max())
    np.testing.assert_allclose(Ur.T @ Gi @ Ur, np.eye(lr.shape[0]), atol=1e-9)
    # rank-4 operator, sketch of 4 columns
    H4 = rng.standard_normal((9, 4)) @ rng.standard_normal((4, Gamma.shape[0]))
    l4, _ = ghep.ghep_exact(H4, R, Gamma, rel_tol=1e-10)
    assert l4.shape[0] == 4
    lr4, _ = ghep.ghep_randomized(H4, R, Gamma, rng.standard_normal((Gamma.shape[0], 4)), 4)
    np.testing.assert_allclose(lr4, l4, rtol=1e-8)


def test_randomized_ghep_ritz_bounds():
    """k + p < rank: Rayleigh-Ritz values are lower bounds of the exact
    eigenvalues and, with eps = |(I - Q Q^T B) B^-1 A|_B, |lam - lam~| <= 2 eps
    (App. B's bound)."""
    rng = np.random.default_rng(34)
    Gamma, H, R = _ghep_problem(rng, N=60, m=30)
    lam, _ = ghep.ghep_exact(H, R, Gamma)
    k, p = 6, 4
    Om = rng.standard_normal((Gamma.shape[0], k + p))
    lr, Ur = ghep.ghep_randomized(H, R, Gamma, Om, k)
    assert np.all(lr <= lam[:k] * (1 + 1e-12))
    # eps from the B-orthonormal basis of the sketch (Q = Gamma Qhat, Q^T B Q = I)
    A = H.T @ (H / R[:, None])
    Qh, _ = ghep.mgs_qr_weighted(A @ Om, Gamma)
    Q = Gamma @ Qh
    B = np.linalg.inv(Gamma)
    C = Gamma @ A
    Eop = (np.eye(Gamma.shape[0]) - Q @ Q.T @ B) @ C
    ev, V = np.linalg.eigh(B)
    Bh = (V * np.sqrt(ev)) @ V.T
    Bmh = (V / np.sqrt(ev)) @ V.T
    eps = np.linalg.norm(Bh @ Eop @ Bmh, 2)
    assert np.all(np.abs(lam[:k] - lr) <= 2 * eps * (1 + 1e-9))


def test_randomized_ghep_filter_is_o1_when_sketch_spans_and_information_form_otherwise():
    """The filter with the randomized GHEP equals O1 when the sketch spans the
    range of H^T R^-1 H (k + p = m); with fewer modes its covariance equals
    the information form with the rank-k data term (scipy inverse), and its
    mean is O1's mean given the same predicted covariance."""
    rng = np.random.default_rng(35)
    N, ms = 30, [6, 6, 6]
    Gamma, steps = _random_problem(rng, N, ms)
    Om = rng.standard_normal((N, 6))
    a = kalman.kf_dense(Gamma, steps)
    b = kalman.kf_dense_randomized_ghep(Gamma, steps, Om, 6)
    for x, y in zip(a, b):
        np.testing.assert_allclose(y["Sigma"], x["Sigma"], rtol=1e-8, atol=1e-10)
        np.testing.assert_allclose(y["s"], x["s"], rtol=1e-8, atol=1e-10)
    k = 3
    c = kalman.kf_dense_randomized_ghep(Gamma, steps[:1], Om[:, :5], k)
    lam, U = ghep.ghep_randomized(steps[0][1], steps[0][2], Gamma, Om[:, :5], k)
    Gi = np.linalg.inv(Gamma)
    info = np.linalg.inv(Gamma) + Gi @ (U * lam) @ U.T @ Gi
    np.testing.assert_allclose(c[0]["Sigma"], np.linalg.inv(info), rtol=1e-8, atol=1e-10)
    np.testing.assert_allclose(c[0]["s"], a[0]["s"], rtol=1e-12, atol=1e-14)
