"""FP64 parity of the compressed operator and of the rank control.

1. Compressed Gamma_H (eta = 1, ACA 1e-8): the filter on the GPU computes the
   Kalman filter of the covariance Gamma_H that the H-matrix represents, so it
   is compared with the dense filter O1 run on that same matrix (exported by
   fkf_hmatrix_densify) at relative 1e-10 -- the far-field sweep, its slot
   pairing and the near tiles all enter.  The H-apply itself is compared with
   densify(Gamma_H) X at 1e-13.
2. Rank control (Alg. lowrankaddition step 4): a rank cap r_max below sum m_k
   and the paper's relative tolerance 1e-5 against O1t, the dense filter
   truncated by the same keep rule after every update.  Invariants:
   W^T Gamma^-1 W = I, Sigma symmetric positive definite, r <= r_max.
"""

import numpy as np
import pytest

import synth
from oracle import covariance, kalman
from tests.helpers import TINY, lib, rel_err, run_filter, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fkf():
    from paper_1405_2276_gb300 import build

    build()
    return lib()


def _destroy(fkf, ctx, hm, f):
    fkf.fkf_filter_destroy(f)
    fkf.fkf_hmatrix_destroy(hm)
    fkf.fkf_destroy(ctx)


def _compare(got, ref, G, bound, check_sigma=True):
    worst = 0.0
    for k, (a, b) in enumerate(zip(got, ref)):
        es, ev = rel_err(a["s"], b["s"]), rel_err(a["var"], b["var"])
        en = abs(a["nll"] - b["nll"]) / abs(b["nll"])
        worst = max(worst, es, ev, en)
        assert es < bound and ev < bound and en < bound, (k, es, ev, en)
        if check_sigma and "W" in a:
            Sig = a["alpha"] * G - (a["W"] * a["D"]) @ a["W"].T
            esig = rel_err(Sig, b["Sigma"])
            worst = max(worst, esig)
            assert esig < bound, (k, esig)
    return worst


@pytest.mark.parametrize("grid,leaf", [((32, 32), 64), ((48, 40), 32)])
def test_compressed_apply_matches_densified_operator(fkf, grid, leaf):
    import torch

    pts = synth.grid_points_2d(*grid)
    n = pts.shape[0]
    ctx = fkf.fkf_create(0)
    hm = fkf.fkf_hmatrix_build(ctx, pts, 1.5, 0.2, 1.0, leaf=leaf, eta=1.0, aca_tol=1e-8, k_cap=32)
    assert fkf.fkf_hmatrix_info(hm)["n_far"] > 0
    D = fkf.fkf_hmatrix_densify(hm, n)
    rng = np.random.default_rng(61)
    for ncols in (1, 33, 256):
        X = rng.standard_normal((n, ncols))
        Xt = torch.from_numpy(X).cuda()
        Yt = torch.empty_like(Xt)
        fkf.fkf_hmatrix_apply(hm, Xt, Yt)
        err = rel_err(Yt.cpu().numpy(), D @ X)
        print(f"{grid} leaf {leaf}: apply vs densified Gamma_H, {ncols} columns: {err:.2e}")
        assert err < 1e-13
    fkf.fkf_hmatrix_destroy(hm)
    fkf.fkf_destroy(ctx)


def test_compressed_filter_fixed_operator_matches_dense_kf_on_gamma_h(fkf):
    wl = workload(TINY)
    pts = wl["points"]
    n = pts.shape[0]
    kern = (TINY["nu"], TINY["ell"], TINY["sigma2"])
    ctx = fkf.fkf_create(0)
    hm = fkf.fkf_hmatrix_build(ctx, pts, *kern, leaf=64, eta=1.0, aca_tol=1e-8, k_cap=32)
    assert fkf.fkf_hmatrix_info(hm)["n_far"] > 0
    GH = fkf.fkf_hmatrix_densify(hm, n)
    np.testing.assert_array_equal(GH, GH.T)
    Hd = synth.csr_to_dense(wl["H"])
    K = wl["y"].shape[0]
    ref = kalman.kf_dense(GH, [(wl["y"][k], Hd, TINY["noise"]) for k in range(K)])
    sg = [(wl["y"][k], wl["H"], TINY["noise"]) for k in range(K)]
    got, _, _, f = run_filter(pts, kern, sg, precision=0, want_W=True, ctx=ctx, hmat=hm)
    worst = _compare(got, ref, GH, 1e-10)
    print(f"compressed Gamma_H, fixed operator, {K} steps vs O1(Gamma_H): worst {worst:.2e}")
    assert fkf.fkf_filter_orthonormality(f) < 1e-9
    _destroy(fkf, ctx, hm, f)


def _varying(seed, nx, ny, ms):
    rng = np.random.default_rng(seed)
    pts = synth.grid_points_2d(nx, ny)
    ops = synth.varying_ray_operators(rng, nx, ny, ms)
    truth = synth.random_walk_truth(rng, (nx, ny), len(ms), 0.2, 1.0)
    ys = [synth.measurements(rng, h, truth[k], 1e-4) for k, h in enumerate(ops)]
    return pts, ops, ys


def test_compressed_filter_time_varying_operators_match_dense_kf_on_gamma_h(fkf):
    """48 x 40 grid, leaf 32, a new ray set every step (rank growth: the
    orthonormalisation and the merge run on the compressed operator)."""
    ms = [6, 14, 9, 20, 11]
    pts, ops, ys = _varying(synth.BASE_SEED + 201, 48, 40, ms)
    n = pts.shape[0]
    kern = (1.5, 0.15, 1.0)
    ctx = fkf.fkf_create(0)
    hm = fkf.fkf_hmatrix_build(ctx, pts, *kern, leaf=32, eta=1.0, aca_tol=1e-8, k_cap=32)
    assert fkf.fkf_hmatrix_info(hm)["n_far"] > 0
    GH = fkf.fkf_hmatrix_densify(hm, n)
    ref = kalman.kf_dense(GH, [(ys[k], synth.csr_to_dense(ops[k]), 1e-4) for k in range(len(ms))])
    sg = [(ys[k], ops[k], 1e-4) for k in range(len(ms))]
    got, _, _, f = run_filter(pts, kern, sg, precision=0, want_W=True, ctx=ctx, hmat=hm, m_max=max(ms),
                              r_max=sum(ms))
    worst = _compare(got, ref, GH, 1e-10)
    assert got[-1]["r"] > max(ms)
    print(f"compressed Gamma_H, new operator every step: worst {worst:.2e}, final rank {got[-1]['r']}")
    _destroy(fkf, ctx, hm, f)


def _check_invariants(fkf, f, rec, G):
    assert fkf.fkf_filter_orthonormality(f) < 1e-9
    Sig = rec["alpha"] * G - (rec["W"] * rec["D"]) @ rec["W"].T
    np.testing.assert_allclose(Sig, Sig.T, atol=1e-12 * np.abs(Sig).max())
    assert np.linalg.eigvalsh(0.5 * (Sig + Sig.T)).min() > 0


@pytest.mark.parametrize("r_max,trunc_tol", [(24, 1e-12), (40, 1e-12), (400, 1e-5)])
def test_rank_control_matches_truncated_dense_kf(fkf, r_max, trunc_tol):
    """Time-varying rays with sum m_k = 72: a rank cap below it (the partial
    eigensolve of the merge keeps the r_max largest pairs) and the paper's
    relative truncation 1e-5 (Sec. 4.2), each against O1t."""
    ms = [5, 12, 7, 20, 9, 16, 3]
    pts, ops, ys = _varying(synth.BASE_SEED + 100, 24, 24, ms)
    kern = (1.5, 0.25, 1.0)
    G = covariance.dense_gamma(pts, *kern)
    so = [(ys[k], synth.csr_to_dense(ops[k]), 1e-4) for k in range(len(ms))]
    ref = kalman.kf_dense_truncated(G, so, r_max=r_max, trunc_tol=trunc_tol)
    sg = [(ys[k], ops[k], 1e-4) for k in range(len(ms))]
    got, ctx, hm, f = run_filter(pts, kern, sg, precision=0, eta=0.0, leaf=32, want_W=True, m_max=max(ms),
                                 r_max=r_max, trunc_tol=trunc_tol)
    ranks = [g["r"] for g in got]
    assert ranks == [q["r"] for q in ref], (ranks, [q["r"] for q in ref])
    assert max(ranks) <= r_max
    if trunc_tol > 1e-10 or r_max < sum(ms):
        assert ranks[-1] < sum(ms)  # the rank control really acted
    for a, b in zip(got, ref):
        # the merge eigensolve is backward stable: each weight carries an absolute
        # error of order eps times the largest merged eigenvalue
        np.testing.assert_allclose(np.sort(a["D"])[::-1], b["d"], rtol=1e-9, atol=1e-9 * b["d"][0])
    worst = _compare(got, ref, G, 1e-9)
    print(f"rank control r_max={r_max} trunc_tol={trunc_tol:g}: ranks {ranks}, worst {worst:.2e}")
    _check_invariants(fkf, f, got[-1], G)
    _destroy(fkf, ctx, hm, f)
