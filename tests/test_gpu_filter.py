"""Filter steps on the GPU (through the C-ABI) against the oracle's dense
Kalman filter (O1) and the fixed-H cross-covariance recursion (O2).

Tolerances:
  * FP64 path with Gamma_H = Gamma (eta = 0, every block dense): relative
    1e-10 on s_hat, diag(Sigma), NLL and the full Sigma (the only differences
    are rounding orders);
  * FP64 path with a compressed Gamma_H (ACA tolerance tol): the oracle uses
    the exact Gamma, so the bound is tol times the filter's sensitivity to a
    relative perturbation of Gamma, estimated by the oracle itself (perturb
    Gamma, rerun O1), times a safety factor of 100;
  * FP32 path: its error against the oracle is reported and bounded loosely.
"""

import numpy as np
import pytest

import synth
from oracle import covariance, kalman, uq
from tests.helpers import TINY, lib, rel_err, run_filter, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fkf():
    from paper_1405_2276_gb300 import build

    build()
    return lib()


def _tiny(steps=None):
    wl = workload(TINY, steps)
    pts = wl["points"]
    G = covariance.dense_gamma(pts, TINY["nu"], TINY["ell"], TINY["sigma2"])
    steps_gpu = [(wl["y"][k], wl["H"], TINY["noise"]) for k in range(wl["y"].shape[0])]
    Hd = synth.csr_to_dense(wl["H"])
    steps_o = [(wl["y"][k], Hd, TINY["noise"]) for k in range(wl["y"].shape[0])]
    return wl, pts, G, steps_gpu, steps_o


KERN = (TINY["nu"], TINY["ell"], TINY["sigma2"])


def test_fp64_exact_gamma_matches_dense_kf(fkf):
    wl, pts, G, sg, so = _tiny()
    ref = kalman.kf_dense(G, so)
    got, ctx, hm, f = run_filter(pts, KERN, sg, precision=0, eta=0.0, want_W=True)
    m = wl["H"].nrows
    for k, (a, b) in enumerate(zip(got, ref)):
        assert a["alpha"] == k + 1
        assert 0 < a["r"] <= m
        assert rel_err(a["s"], b["s"]) < 1e-10, k
        assert rel_err(a["var"], b["var"]) < 1e-10, k
        assert abs(a["nll"] - b["nll"]) < 1e-10 * abs(b["nll"]), k
        # full covariance alpha Gamma - W D W^T  (fixes span(W), basis-free)
        Sig = a["alpha"] * G - (a["W"] * a["D"]) @ a["W"].T
        assert rel_err(Sig, b["Sigma"]) < 1e-10, k
        assert np.all(a["D"] > 0) and np.all(a["D"] < a["alpha"])
    # W^T Gamma^-1 W = I
    W = got[-1]["W"]
    np.testing.assert_allclose(W.T @ np.linalg.solve(G, W), np.eye(W.shape[1]), atol=1e-8)
    assert fkf.fkf_filter_orthonormality(f) < 1e-9
    fkf.fkf_filter_destroy(f)
    fkf.fkf_hmatrix_destroy(hm)
    fkf.fkf_destroy(ctx)


def _sensitivity(G, so, delta=1e-8, seed=0):
    """Oracle-only estimate of the relative change of O1's outputs per unit
    relative symmetric perturbation of Gamma."""
    rng = np.random.default_rng(seed)
    E = rng.standard_normal(G.shape)
    E = 0.5 * (E + E.T)
    E *= delta * np.linalg.norm(G) / np.linalg.norm(E)
    a = kalman.kf_dense(G, so, keep_cov=False)
    b = kalman.kf_dense(G + E, so, keep_cov=False)
    amp = 0.0
    for x, y in zip(a, b):
        amp = max(amp, rel_err(y["s"], x["s"]) / delta, rel_err(y["var"], x["var"]) / delta)
    return amp


def test_fp64_compressed_gamma_within_compression_bound(fkf):
    wl, pts, G, sg, so = _tiny()
    ref = kalman.kf_dense(G, so, keep_cov=False)
    tol = 1e-8
    amp = _sensitivity(G, so)
    bound = 100 * amp * tol
    got, ctx, hm, f = run_filter(pts, KERN, sg, precision=0, eta=1.0, aca_tol=tol, leaf=64)
    assert fkf.fkf_hmatrix_info(hm)["n_far"] > 0
    worst = max(max(rel_err(a["s"], b["s"]), rel_err(a["var"], b["var"])) for a, b in zip(got, ref))
    print(f"compressed FP64 vs exact-Gamma oracle: worst rel err {worst:.3e} (bound {bound:.3e}, amp {amp:.1f})")
    assert worst < bound
    fkf.fkf_filter_destroy(f)
    fkf.fkf_hmatrix_destroy(hm)
    fkf.fkf_destroy(ctx)


def test_time_varying_operators_match_dense_kf(fkf):
    """A new H_k (and a new m_k) every step: the rank grows as sum m_k and the
    general path (orthonormalisation + merge) is exercised."""
    rng = np.random.default_rng(synth.BASE_SEED + 100)
    nx = ny = 24
    pts = synth.grid_points_2d(nx, ny)
    ms = [5, 12, 7, 20, 9, 16, 3]
    ops = synth.varying_ray_operators(rng, nx, ny, ms)
    truth = synth.random_walk_truth(rng, (nx, ny), len(ms), 0.2, 1.0)
    ys = [synth.measurements(rng, h, truth[k], 1e-4) for k, h in enumerate(ops)]
    G = covariance.dense_gamma(pts, 1.5, 0.25, 1.0)
    so = [(ys[k], synth.csr_to_dense(ops[k]), 1e-4) for k in range(len(ms))]
    ref = kalman.kf_dense(G, so)
    sg = [(ys[k], ops[k], 1e-4) for k in range(len(ms))]
    got, ctx, hm, f = run_filter(pts, (1.5, 0.25, 1.0), sg, precision=0, eta=0.0, leaf=32, want_W=True,
                                 m_max=max(ms), r_max=sum(ms))
    for k, (a, b) in enumerate(zip(got, ref)):
        assert a["r"] <= sum(ms[: k + 1])
        assert rel_err(a["s"], b["s"]) < 1e-10, k
        assert rel_err(a["var"], b["var"]) < 1e-10, k
        Sig = a["alpha"] * G - (a["W"] * a["D"]) @ a["W"].T
        assert rel_err(Sig, b["Sigma"]) < 1e-10, k
        assert abs(a["nll"] - b["nll"]) < 1e-10 * abs(b["nll"]), k
    assert got[-1]["r"] > max(ms)  # rank really grew
    fkf.fkf_filter_destroy(f)
    fkf.fkf_hmatrix_destroy(hm)
    fkf.fkf_destroy(ctx)


def test_diagonal_R_and_zero_rows(fkf):
    """Per-measurement noise variances and an all-zero row of H."""
    rng = np.random.default_rng(5)
    nx, ny = 16, 12
    pts = synth.grid_points_2d(nx, ny)
    ops = synth.varying_ray_operators(rng, nx, ny, [6, 6, 6])
    # zero out row 2 of the second operator
    h = ops[1]
    keep = np.ones(h.nnz, bool)
    keep[h.rowptr[2] : h.rowptr[3]] = False
    cnt = np.diff(h.rowptr)
    cnt[2] = 0
    ops[1] = synth.Csr(np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64), h.col[keep], h.val[keep], h.ncols)
    Rs = [rng.uniform(5e-5, 5e-4, 6) for _ in range(3)]
    ys = [rng.standard_normal(6) for _ in range(3)]
    G = covariance.dense_gamma(pts, 0.5, 0.3, 1.5)
    ref = kalman.kf_dense(G, [(ys[k], synth.csr_to_dense(ops[k]), Rs[k]) for k in range(3)])
    got, ctx, hm, f = run_filter(pts, (0.5, 0.3, 1.5), [(ys[k], ops[k], Rs[k]) for k in range(3)], eta=0.0, leaf=16,
                                 m_max=6, r_max=18)
    for a, b in zip(got, ref):
        assert rel_err(a["s"], b["s"]) < 1e-10
        assert rel_err(a["var"], b["var"]) < 1e-10
        assert abs(a["nll"] - b["nll"]) < 1e-10 * abs(b["nll"])
    fkf.fkf_filter_destroy(f)
    fkf.fkf_hmatrix_destroy(hm)
    fkf.fkf_destroy(ctx)


def test_fp32_path_error_vs_oracle(fkf):
    wl, pts, G, sg, so = _tiny()
    ref = kalman.kf_dense(G, so, keep_cov=False)
    got, ctx, hm, f = run_filter(pts, KERN, sg, precision=1, eta=1.0, aca_tol=1e-8)
    es = max(rel_err(a["s"], b["s"]) for a, b in zip(got, ref))
    ev = max(rel_err(a["var"], b["var"]) for a, b in zip(got, ref))
    print(f"FP32 path vs FP64 oracle: s_hat rel err {es:.3e}, variance rel err {ev:.3e}")
    # measured about 1e-5 (s_hat) and 3e-6 (variance): bound at 10-20x that
    assert es < 2e-4 and ev < 2e-4
    fkf.fkf_filter_destroy(f)
    fkf.fkf_hmatrix_destroy(hm)
    fkf.fkf_destroy(ctx)


def test_realization_variance_and_scalars(fkf):
    import torch

    wl, pts, G, sg, so = _tiny(steps=4)
    ref = kalman.kf_dense(G, so)
    got, ctx, hm, f = run_filter(pts, KERN, sg, precision=0, eta=0.0)
    n = pts.shape[0]
    Sig = ref[-1]["Sigma"]
    alpha = got[-1]["alpha"]
    rng = np.random.default_rng(9)
    L = np.linalg.cholesky(G)
    a = L @ rng.standard_normal((n, 16))
    a_t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = torch.empty_like(a_t)
    fkf.fkf_conditional_realization(f, a_t, out)
    x_ref = uq.realization(ref[-1]["s"], Sig, G, alpha, a)
    assert rel_err(out.cpu().numpy(), x_ref) < 1e-9
    ent, tr = fkf.fkf_uncertainty_scalars(f)
    assert abs(ent - uq.relative_entropy(Sig, G)) < 1e-8 * abs(ent)
    assert abs(tr - uq.a_optimality_identity(Sig)) < 1e-10 * abs(tr)
    fkf.fkf_filter_destroy(f)
    fkf.fkf_hmatrix_destroy(hm)
    fkf.fkf_destroy(ctx)


def test_checkpoint_restore_is_bitwise(fkf, tmp_path):
    wl, pts, G, sg, so = _tiny()
    ctx = fkf.fkf_create(0)
    hm = fkf.fkf_hmatrix_build(ctx, pts, *KERN, leaf=64, eta=1.0, aca_tol=1e-8)
    n = pts.shape[0]
    m = wl["H"].nrows

    def step(f, k):
        h = wl["H"]
        return fkf.fkf_filter_step(f, wl["y"][k], m, h.rowptr, h.col, h.val, None, TINY["noise"])

    f1 = fkf.fkf_filter_create(hm, None, 0.0, 1e-12, m, 2 * m)
    for k in range(5):
        step(f1, k)
    path = str(tmp_path / "ck.bin")
    fkf.fkf_filter_checkpoint(f1, path)
    n1 = [step(f1, k) for k in range(5, 8)]
    s1 = fkf.fkf_filter_get(f1, n)
    f2 = fkf.fkf_filter_create(hm, None, 0.0, 1e-12, m, 2 * m)
    fkf.fkf_filter_restore(f2, path)
    n2 = [step(f2, k) for k in range(5, 8)]
    s2 = fkf.fkf_filter_get(f2, n)
    assert n1 == n2
    np.testing.assert_array_equal(s1["s"], s2["s"])
    np.testing.assert_array_equal(s1["D"], s2["D"])
    assert s1["alpha"] == s2["alpha"] == 8
    for f in (f1, f2):
        fkf.fkf_filter_destroy(f)
    fkf.fkf_hmatrix_destroy(hm)
    fkf.fkf_destroy(ctx)


def test_invalid_inputs_leave_state_unchanged(fkf):
    wl, pts, G, sg, so = _tiny(steps=3)
    ctx = fkf.fkf_create(0)
    hm = fkf.fkf_hmatrix_build(ctx, pts, *KERN, leaf=64, eta=0.0)
    n = pts.shape[0]
    h = wl["H"]
    m = h.nrows
    f = fkf.fkf_filter_create(hm, None, 0.0, 1e-12, m, 2 * m)
    fkf.fkf_filter_step(f, wl["y"][0], m, h.rowptr, h.col, h.val, None, 1e-4)
    before = fkf.fkf_filter_get(f, n)
    bad_col = h.col.copy()
    bad_col[3] = n + 5
    cases = [
        dict(col=bad_col, R=None, rs=1e-4, m=m),
        dict(col=h.col, R=None, rs=-1.0, m=m),
        dict(col=h.col, R=np.full(m, 0.0), rs=0.0, m=m),
        dict(col=h.col, R=None, rs=1e-4, m=m + 1),
    ]
    for c in cases:
        with pytest.raises(fkf.FkfError) as e:
            rowptr = h.rowptr if c["m"] == m else np.concatenate([h.rowptr, h.rowptr[-1:]])
            fkf.fkf_filter_step(f, np.zeros(c["m"]), c["m"], rowptr, c["col"], h.val, c["R"], c["rs"])
        assert e.value.status == fkf.FKF_EINVAL
        after = fkf.fkf_filter_get(f, n)
        np.testing.assert_array_equal(after["s"], before["s"])
        np.testing.assert_array_equal(after["D"], before["D"])
        assert after["alpha"] == before["alpha"] and after["r"] == before["r"]
    fkf.fkf_filter_destroy(f)
    fkf.fkf_hmatrix_destroy(hm)
    fkf.fkf_destroy(ctx)


def test_refresh_keeps_covariance(fkf):
    """A manual refresh (W <- Gamma_H X, re-orthonormalised) after 6 steps:
    the state still equals the dense oracle's posterior."""
    wl, pts, G, sg, so = _tiny(steps=6)
    ref = kalman.kf_dense(G, so)
    got, ctx, hm, f = run_filter(pts, KERN, sg, precision=0, eta=0.0)
    import torch

    n = pts.shape[0]
    fkf.fkf_filter_refresh(f)
    v1 = torch.empty(n, dtype=torch.float64, device="cuda")
    fkf.fkf_variance(f, v1)
    assert rel_err(v1.cpu().numpy(), ref[-1]["var"]) < 1e-10
    st = fkf.fkf_filter_get(f, n)
    W = torch.empty((n, st["r"]), dtype=torch.float64, device="cuda")
    fkf.fkf_filter_get(f, n, want_s=False, want_D=False, W=W)
    W = W.cpu().numpy()
    assert rel_err(st["alpha"] * G - (W * st["D"]) @ W.T, ref[-1]["Sigma"]) < 1e-10
    assert fkf.fkf_filter_orthonormality(f) < 1e-10
    fkf.fkf_filter_destroy(f)
    fkf.fkf_hmatrix_destroy(hm)
    fkf.fkf_destroy(ctx)


def test_scheduled_refresh_with_rank_above_m_max_matches_dense_kf(fkf):
    """S10 scheduled every 2 steps on the FP64 path with a new operator every
    step, so the rank (up to sum m_k = 72) exceeds m_max = 20 and the refresh
    needs its own N x r scratch; every step against O1 at 1e-10."""
    import torch

    rng = np.random.default_rng(synth.BASE_SEED + 100)
    nx = ny = 24
    pts = synth.grid_points_2d(nx, ny)
    ms = [5, 12, 7, 20, 9, 16, 3]
    ops = synth.varying_ray_operators(rng, nx, ny, ms)
    truth = synth.random_walk_truth(rng, (nx, ny), len(ms), 0.2, 1.0)
    ys = [synth.measurements(rng, h, truth[k], 1e-4) for k, h in enumerate(ops)]
    G = covariance.dense_gamma(pts, 1.5, 0.25, 1.0)
    ref = kalman.kf_dense(G, [(ys[k], synth.csr_to_dense(ops[k]), 1e-4) for k in range(len(ms))])
    n = pts.shape[0]
    ctx = fkf.fkf_create(0)
    hm = fkf.fkf_hmatrix_build(ctx, pts, 1.5, 0.25, 1.0, leaf=32, eta=0.0)
    f = fkf.fkf_filter_create(hm, None, 0.0, 1e-12, max(ms), sum(ms))
    fkf.fkf_filter_set_refresh(f, 2)
    for k, h in enumerate(ops):
        nll = fkf.fkf_filter_step(f, ys[k], h.nrows, h.rowptr, h.col, h.val, None, 1e-4)
        st = fkf.fkf_filter_get(f, n)
        W = torch.empty((n, st["r"]), dtype=torch.float64, device="cuda")
        fkf.fkf_filter_get(f, n, want_s=False, want_D=False, W=W)
        W = W.cpu().numpy()
        assert rel_err(st["s"], ref[k]["s"]) < 1e-10, k
        assert rel_err(st["alpha"] * G - (W * st["D"]) @ W.T, ref[k]["Sigma"]) < 1e-10, k
        assert abs(nll - ref[k]["nll"]) < 1e-10 * abs(ref[k]["nll"]), k
        if (k + 1) % 2 == 0:
            assert fkf.fkf_filter_orthonormality(f) < 1e-11, k
    assert st["r"] > max(ms)
    fkf.fkf_filter_destroy(f)
    fkf.fkf_hmatrix_destroy(hm)
    fkf.fkf_destroy(ctx)


def test_scheduled_refresh_fp32_matches_dense_kf(fkf):
    """S10 on the FP32 path (the state the refresh is for): refresh every 3
    steps, compared with O1 on s_hat and diag(Sigma)."""
    wl, pts, G, sg, so = _tiny()
    ref = kalman.kf_dense(G, so, keep_cov=False)
    got, ctx, hm, f = run_filter(pts, KERN, sg, precision=1, eta=1.0, aca_tol=1e-8, refresh_every=3)
    es = max(rel_err(a["s"], b["s"]) for a, b in zip(got, ref))
    ev = max(rel_err(a["var"], b["var"]) for a, b in zip(got, ref))
    print(f"FP32 path with refresh every 3 steps vs FP64 oracle: s_hat {es:.3e}, var {ev:.3e}")
    assert es < 2e-4 and ev < 2e-4
    fkf.fkf_filter_destroy(f)
    fkf.fkf_hmatrix_destroy(hm)
    fkf.fkf_destroy(ctx)


def test_fixed_geometry_rank_stays_at_m(fkf):
    wl, pts, G, sg, so = _tiny()
    got, ctx, hm, f = run_filter(pts, KERN, sg, precision=0, eta=1.0, aca_tol=1e-8, want_var=False)
    m = wl["H"].nrows
    assert all(g["r"] <= m for g in got)
    fkf.fkf_filter_destroy(f)
    fkf.fkf_hmatrix_destroy(hm)
    fkf.fkf_destroy(ctx)


def test_kept_basis_steps_then_new_operator_match_dense_kf(fkf):
    """A repeated operator brings no information outside span(W): the basis is
    kept and the (then non-diagonal) weight is updated in information form,
    several steps in a row with no observation in between; a new operator
    then forces the merge path.  Everything against the dense oracle."""
    rng = np.random.default_rng(synth.BASE_SEED + 7)
    nx = ny = 20
    pts = synth.grid_points_2d(nx, ny)
    p0, p1 = synth.cross_well_geometry_2d(6, 4)
    Ha = synth.trace_rays_2d(nx, ny, p0, p1)
    Hb = synth.varying_ray_operators(rng, nx, ny, [15])[0]
    seq = [Ha, Ha, Ha, Ha, Hb, Ha, Ha, Ha]
    ys = [rng.standard_normal(h.nrows) * 0.3 for h in seq]
    G = covariance.dense_gamma(pts, 1.5, 0.25, 1.0)
    ref = kalman.kf_dense(G, [(ys[k], synth.csr_to_dense(h), 1e-4) for k, h in enumerate(seq)])
    ctx = fkf.fkf_create(0)
    hm = fkf.fkf_hmatrix_build(ctx, pts, 1.5, 0.25, 1.0, leaf=32, eta=0.0)
    f = fkf.fkf_filter_create(hm, None, 0.0, 1e-12, 24, 48)
    paths = []
    for k, h in enumerate(seq):
        nll = fkf.fkf_filter_step(f, ys[k], h.nrows, h.rowptr, h.col, h.val, None, 1e-4)
        assert abs(nll - ref[k]["nll"]) < 1e-10 * abs(ref[k]["nll"]), k
        paths.append(fkf.fkf_filter_get_stats(f)["last_path"])
    assert paths == [0, 1, 1, 1, 0, 1, 1, 1]
    assert fkf.fkf_filter_get_stats(f)["diagonal"] == 0
    assert fkf.fkf_library_call_count(ctx) == len(seq)  # one vendor routine per step: the innovation solve
    import torch

    n = pts.shape[0]
    st = fkf.fkf_filter_get(f, n)
    assert fkf.fkf_filter_get_stats(f)["diagonal"] == 1
    W = torch.empty((n, st["r"]), dtype=torch.float64, device="cuda")
    fkf.fkf_filter_get(f, n, want_s=False, want_D=False, W=W)
    W = W.cpu().numpy()
    Sig = st["alpha"] * G - (W * st["D"]) @ W.T
    assert rel_err(st["s"], ref[-1]["s"]) < 1e-10
    assert rel_err(Sig, ref[-1]["Sigma"]) < 1e-10
    np.testing.assert_allclose(W.T @ np.linalg.solve(G, W), np.eye(W.shape[1]), atol=1e-8)
    fkf.fkf_filter_destroy(f)
    fkf.fkf_hmatrix_destroy(hm)
    fkf.fkf_destroy(ctx)


def test_innovation_solve_ragged_blocks_match_dense_kf(fkf):
    """m = 97 and 161 rays: the blocked Cholesky factorisation of the
    innovation system (bordered on the kept-basis steps) runs over several
    32-row blocks with a ragged last block; NLL and mean against the dense
    oracle at 1e-10, and exactly one vendor routine (the innovation solve) per
    step."""
    rng = np.random.default_rng(synth.BASE_SEED + 21)
    nx = ny = 20
    pts = synth.grid_points_2d(nx, ny)
    Ha, Hb = synth.varying_ray_operators(rng, nx, ny, [97, 161])
    seq = [Ha, Ha, Hb, Hb]
    ys = [rng.standard_normal(h.nrows) * 0.3 for h in seq]
    G = covariance.dense_gamma(pts, 1.5, 0.25, 1.0)
    ref = kalman.kf_dense(G, [(ys[k], synth.csr_to_dense(h), 1e-4) for k, h in enumerate(seq)])
    ctx = fkf.fkf_create(0)
    hm = fkf.fkf_hmatrix_build(ctx, pts, 1.5, 0.25, 1.0, leaf=32, eta=0.0)
    f = fkf.fkf_filter_create(hm, None, 0.0, 1e-12, 161, 400)
    for k, h in enumerate(seq):
        nll = fkf.fkf_filter_step(f, ys[k], h.nrows, h.rowptr, h.col, h.val, None, 1e-4)
        assert abs(nll - ref[k]["nll"]) < 1e-10 * abs(ref[k]["nll"]), k
    n = pts.shape[0]
    st = fkf.fkf_filter_get(f, n)
    assert rel_err(st["s"], ref[-1]["s"]) < 1e-10
    assert fkf.fkf_library_call_count(ctx) == len(seq)
    fkf.fkf_filter_destroy(f)
    fkf.fkf_hmatrix_destroy(hm)
    fkf.fkf_destroy(ctx)


@pytest.mark.parametrize("device_inputs", [False, True])
def test_fixed_h_fast_path_reuses_products_exactly(fkf, device_inputs):
    """FKF_STEP_ALLOW_FIXED_H with a repeated operator: after the first
    kept-basis step the products G = Gamma_H H^T and H [W G] are reused (path
    3); every result equals the run that recomputes them (the reused arrays
    are the ones the recomputation would produce bit for bit).  A changed H
    entry is detected and recomputed."""
    import torch

    rng = np.random.default_rng(synth.BASE_SEED + 11)
    nx = ny = 20
    pts = synth.grid_points_2d(nx, ny)
    p0, p1 = synth.cross_well_geometry_2d(6, 4)
    Ha = synth.trace_rays_2d(nx, ny, p0, p1)
    ys = [rng.standard_normal(Ha.nrows) * 0.3 for _ in range(6)]
    n = pts.shape[0]

    def arrays(h, y):
        if not device_inputs:
            return y, h.rowptr, h.col, h.val
        return tuple(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (y, h.rowptr, h.col, h.val))

    def run(allow, seq):
        ctx = fkf.fkf_create(0)
        hm = fkf.fkf_hmatrix_build(ctx, pts, 1.5, 0.25, 1.0, leaf=32, eta=1.0, aca_tol=1e-10)
        f = fkf.fkf_filter_create(hm, None, 0.0, 1e-12, 24, 48)
        flags = (fkf.FKF_STEP_ALLOW_FIXED_H if allow else 0) | (fkf.FKF_STEP_INPUTS_ON_DEVICE if device_inputs else 0)
        nlls, paths = [], []
        for y, h in seq:
            yy, rp, cc, vv = arrays(h, y)
            nlls.append(fkf.fkf_filter_step(f, yy, h.nrows, rp, cc, vv, None, 1e-4, flags=flags))
            paths.append(fkf.fkf_filter_get_stats(f)["last_path"])
        st = fkf.fkf_filter_get(f, n)
        fkf.fkf_filter_destroy(f)
        fkf.fkf_hmatrix_destroy(hm)
        fkf.fkf_destroy(ctx)
        return nlls, paths, st

    seq = [(y, Ha) for y in ys]
    a_nll, a_paths, a_st = run(False, seq)
    b_nll, b_paths, b_st = run(True, seq)
    assert a_paths == [0, 1, 1, 1, 1, 1]
    assert b_paths == [0, 1, 3, 3, 3, 3]
    assert a_nll == b_nll
    np.testing.assert_array_equal(a_st["s"], b_st["s"])
    np.testing.assert_array_equal(a_st["D"], b_st["D"])
    # one changed value in H: no reuse for that step
    Hc = synth.Csr(Ha.rowptr.copy(), Ha.col.copy(), Ha.val.copy(), Ha.ncols)
    Hc.val[3] *= 1.0 + 1e-12
    c_nll, c_paths, _ = run(True, seq[:3] + [(ys[3], Hc)] + seq[4:])
    assert c_paths[:3] == [0, 1, 3] and c_paths[3] != 3


@pytest.mark.parametrize("precision,eta,bound", [(0, 0.0, 1e-10), (1, 1.0, 5e-3)])
def test_3d_voxels_and_rays_match_dense_kf(fkf, precision, eta, bound):
    """A 3D voxel grid (12 x 10 x 14) with straight rays between lattices on
    two opposite faces (the 3D workload's geometry, small enough for the dense
    oracle): the octree H-matrix and the filter against the dense KF, and 16
    conditional realizations per step through the same path."""
    import torch

    wl = synth.tomography_workload((12, 10, 14), (3, 4), (4, 3), 4, 0.3, 1.0, 1e-4, seed=synth.BASE_SEED + 91)
    pts = wl["points"]
    kern = (0.5, 0.3, 1.0)
    G = covariance.dense_gamma(pts, *kern)
    Hd = synth.csr_to_dense(wl["H"])
    ref = kalman.kf_dense(G, [(wl["y"][k], Hd, 1e-4) for k in range(4)])
    sg = [(wl["y"][k], wl["H"], 1e-4) for k in range(4)]
    got, ctx, hm, f = run_filter(pts, kern, sg, precision=precision, leaf=40, eta=eta, aca_tol=1e-10)
    for a, b in zip(got, ref):
        assert rel_err(a["s"], b["s"]) < bound
        assert rel_err(a["var"], b["var"]) < bound
    n = pts.shape[0]
    L = np.linalg.cholesky(G)
    a = L @ np.random.default_rng(4).standard_normal((n, 16))
    a_t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = torch.empty_like(a_t)
    fkf.fkf_conditional_realization(f, a_t, out)
    x_ref = uq.realization(ref[-1]["s"], ref[-1]["Sigma"], G, got[-1]["alpha"], a)
    assert rel_err(out.cpu().numpy(), x_ref) < (1e-9 if precision == 0 else 5e-3)
    fkf.fkf_filter_destroy(f)
    fkf.fkf_hmatrix_destroy(hm)
    fkf.fkf_destroy(ctx)
