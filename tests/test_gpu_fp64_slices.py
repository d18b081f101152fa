"""FP64 operators on the tensor cores (engine 3: products of 7-bit integer
slices, Ozaki's error-free splitting, FP16 MMAs with exact FP32 sums).

1. The apply against the exact FP64 apply of the same operator (SIMT
   engine 0) and against densify(Gamma_H) X, on grids whose clusters span
   several leaf groups (FP64 partial rows), with ragged column counts and more
   columns than one pass holds.  The slices keep 49 bits of every value
   relative to its row (column) scale: the bound is 1e-12 of max |Y|.
2. The FP64 filter with the engine against the dense Kalman filter O1 on the
   densified Gamma_H at 1e-10 (fixed and time-varying operators), as the
   exact FP64 path is held.
"""

import numpy as np
import pytest

import synth
from oracle import kalman
from tests.helpers import TINY, lib, rel_err, run_filter, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fkf():
    from paper_1405_2276_gb300 import build

    build()
    return lib()


def _apply(fkf, hm, X):
    import torch

    Xt = torch.from_numpy(X).cuda()
    Yt = torch.empty_like(Xt)
    fkf.fkf_hmatrix_apply(hm, Xt, Yt)
    return Yt.cpu().numpy()


@pytest.mark.parametrize("grid,leaf,nu,ell,cols", [
    ((37, 23), 16, 1.5, 0.2, (1, 7, 300)),
    ((64, 48), 32, 0.5, 0.1, (130,)),
    ((128, 96), 64, 0.5, 0.05, (260,)),
])
def test_slice_engine_matches_exact_fp64_apply(fkf, grid, leaf, nu, ell, cols):
    pts = synth.grid_points_2d(*grid)
    n = pts.shape[0]
    ctx = fkf.fkf_create(0)
    hm = fkf.fkf_hmatrix_build(ctx, pts, nu, ell, 1.0, leaf=leaf, eta=1.0, aca_tol=1e-8, k_cap=32, precision=0)
    assert fkf.fkf_hmatrix_info(hm)["n_far"] > 0
    D = fkf.fkf_hmatrix_densify(hm, n) if n <= 8192 else None
    rng = np.random.default_rng(91)
    for ncols in cols:
        X = rng.standard_normal((n, ncols))
        fkf.fkf_hmatrix_set_engine(hm, 0)
        Y0 = _apply(fkf, hm, X)
        fkf.fkf_hmatrix_set_engine(hm, 3)
        assert fkf.fkf_hmatrix_get_engine(hm) == 3
        Y3 = _apply(fkf, hm, X)
        Y3b = _apply(fkf, hm, X)
        np.testing.assert_array_equal(Y3, Y3b)  # deterministic
        err = rel_err(Y3, Y0)
        msg = f"{grid} leaf {leaf}, {ncols} columns: slices vs exact FP64 apply {err:.2e}"
        if D is not None:
            errd = rel_err(Y3, D @ X)
            msg += f", vs densified Gamma_H {errd:.2e}"
            assert errd < 1e-12
        print(msg)
        assert err < 1e-12, msg
    fkf.fkf_hmatrix_destroy(hm)
    fkf.fkf_destroy(ctx)


def test_slice_engine_many_columns_and_passes(fkf):
    """256 x 256 grid, 1100 columns (more than one column pass): sampled rows
    against the exact FP64 apply."""
    import torch

    pts = synth.grid_points_2d(256, 256)
    n = pts.shape[0]
    ctx = fkf.fkf_create(0)
    hm = fkf.fkf_hmatrix_build(ctx, pts, 1.5, 0.1, 1.0, leaf=64, eta=1.0, aca_tol=1e-8, k_cap=32, precision=0)
    rng = np.random.default_rng(92)
    ncols = 1100
    Xt = torch.from_numpy(rng.standard_normal((n, ncols))).cuda()
    Y0 = torch.empty_like(Xt)
    Y3 = torch.empty_like(Xt)
    fkf.fkf_hmatrix_apply(hm, Xt, Y0)
    fkf.fkf_hmatrix_set_engine(hm, 3)
    fkf.fkf_hmatrix_apply(hm, Xt, Y3)
    err = (Y3 - Y0).abs().max().item() / Y0.abs().max().item()
    print(f"256x256, {ncols} columns: slices vs exact FP64 apply {err:.2e}")
    assert err < 5e-12
    del Xt, Y0, Y3
    fkf.fkf_hmatrix_destroy(hm)
    fkf.fkf_destroy(ctx)


def test_engine_rules(fkf):
    pts = synth.grid_points_2d(20, 13)
    ctx = fkf.fkf_create(0)
    h64 = fkf.fkf_hmatrix_build(ctx, pts, 1.5, 0.3, 1.0, leaf=16, precision=0)
    h32 = fkf.fkf_hmatrix_build(ctx, pts, 1.5, 0.3, 1.0, leaf=16, precision=1)
    for h, bad in ((h64, 1), (h64, 2), (h32, 3)):
        with pytest.raises(fkf.FkfError):
            fkf.fkf_hmatrix_set_engine(h, bad)
    fkf.fkf_hmatrix_set_engine(h64, 3)
    fkf.fkf_hmatrix_set_engine(h64, 0)
    assert fkf.fkf_hmatrix_get_engine(h64) == 0
    fkf.fkf_hmatrix_destroy(h64)
    fkf.fkf_hmatrix_destroy(h32)
    fkf.fkf_destroy(ctx)


def test_fp64_filter_on_slice_engine_matches_dense_kf_on_gamma_h(fkf):
    wl = workload(TINY)
    pts = wl["points"]
    n = pts.shape[0]
    kern = (TINY["nu"], TINY["ell"], TINY["sigma2"])
    ctx = fkf.fkf_create(0)
    hm = fkf.fkf_hmatrix_build(ctx, pts, *kern, leaf=64, eta=1.0, aca_tol=1e-8, k_cap=32)
    fkf.fkf_hmatrix_set_engine(hm, 3)
    GH = fkf.fkf_hmatrix_densify(hm, n)
    Hd = synth.csr_to_dense(wl["H"])
    K = wl["y"].shape[0]
    ref = kalman.kf_dense(GH, [(wl["y"][k], Hd, TINY["noise"]) for k in range(K)])
    sg = [(wl["y"][k], wl["H"], TINY["noise"]) for k in range(K)]
    got, _, _, f = run_filter(pts, kern, sg, precision=0, ctx=ctx, hmat=hm)
    worst = 0.0
    for k, (a, b) in enumerate(zip(got, ref)):
        es, ev = rel_err(a["s"], b["s"]), rel_err(a["var"], b["var"])
        en = abs(a["nll"] - b["nll"]) / abs(b["nll"])
        worst = max(worst, es, ev, en)
        assert es < 1e-10 and ev < 1e-10 and en < 1e-10, (k, es, ev, en)
    print(f"FP64 filter on the slice engine, {K} steps vs O1(Gamma_H): worst {worst:.2e}")
    fkf.fkf_filter_destroy(f)
    fkf.fkf_hmatrix_destroy(hm)
    fkf.fkf_destroy(ctx)


def test_fp64_filter_on_slice_engine_time_varying(fkf):
    ms = [6, 14, 9, 20, 11]
    rng = np.random.default_rng(synth.BASE_SEED + 211)
    nx, ny = 48, 40
    pts = synth.grid_points_2d(nx, ny)
    ops = synth.varying_ray_operators(rng, nx, ny, ms)
    truth = synth.random_walk_truth(rng, (nx, ny), len(ms), 0.2, 1.0)
    ys = [synth.measurements(rng, h, truth[k], 1e-4) for k, h in enumerate(ops)]
    n = pts.shape[0]
    kern = (1.5, 0.15, 1.0)
    ctx = fkf.fkf_create(0)
    hm = fkf.fkf_hmatrix_build(ctx, pts, *kern, leaf=32, eta=1.0, aca_tol=1e-8, k_cap=32)
    fkf.fkf_hmatrix_set_engine(hm, 3)
    GH = fkf.fkf_hmatrix_densify(hm, n)
    ref = kalman.kf_dense(GH, [(ys[k], synth.csr_to_dense(ops[k]), 1e-4) for k in range(len(ms))])
    sg = [(ys[k], ops[k], 1e-4) for k in range(len(ms))]
    got, _, _, f = run_filter(pts, kern, sg, precision=0, ctx=ctx, hmat=hm, m_max=max(ms), r_max=sum(ms))
    worst = 0.0
    for k, (a, b) in enumerate(zip(got, ref)):
        es, ev = rel_err(a["s"], b["s"]), rel_err(a["var"], b["var"])
        worst = max(worst, es, ev)
        assert es < 1e-10 and ev < 1e-10, (k, es, ev)
    print(f"FP64 filter on the slice engine, new rays every step vs O1(Gamma_H): worst {worst:.2e}")
    fkf.fkf_filter_destroy(f)
    fkf.fkf_hmatrix_destroy(hm)
    fkf.fkf_destroy(ctx)


@pytest.mark.parametrize("M,N,K,ta,tb,beta", [
    (1, 1, 1, False, False, 0.0),
    (300, 200, 700, False, False, 0.0),
    (129, 65, 1100, True, False, 0.5),
    (257, 130, 33, False, True, -1.0),
    (1024, 1024, 1024, True, True, 0.0),
])
def test_gemm_f64_on_tensor_cores(fkf, M, N, K, ta, tb, beta):
    """fkf_gemm_f64 against numpy's FP64 product: the error of each element
    below 2^-47 of K max_k |a_ik| max_k |b_kj| (plus |beta c_ij|: the slices
    keep 49 bits of every value relative to its row / column scale); rows and
    columns of very different magnitude."""
    import torch

    rng = np.random.default_rng(M * 7 + N * 3 + K)
    Aop = rng.standard_normal((M, K)) * np.exp(rng.uniform(-8, 8, (M, 1)))
    Bop = rng.standard_normal((K, N)) * np.exp(rng.uniform(-8, 8, (1, N)))
    C0 = rng.standard_normal((M, N))
    A = np.ascontiguousarray(Aop.T) if ta else Aop
    B = np.ascontiguousarray(Bop.T) if tb else Bop
    ctx = fkf.fkf_create(0)
    Ct = torch.from_numpy(C0.copy()).cuda()
    fkf.fkf_gemm_f64(ctx, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), Ct, alpha=1.5, beta=beta,
                     trans_a=ta, trans_b=tb)
    ref = 1.5 * (Aop @ Bop) + beta * C0
    scale = 1.5 * K * np.abs(Aop).max(axis=1)[:, None] * np.abs(Bop).max(axis=0)[None, :] + abs(beta) * np.abs(C0)
    err = float(np.max(np.abs(Ct.cpu().numpy() - ref) / scale))
    print(f"gemm {M}x{N}x{K} ta={ta} tb={tb} beta={beta}: max err / (K max|a| max|b|) {err:.2e}")
    assert err < 2.0 ** -47
    fkf.fkf_destroy(ctx)


def test_gemm_f64_rejects_bad_arguments(fkf):
    import torch

    ctx = fkf.fkf_create(0)
    A = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    B = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(fkf.FkfError) as e:  # C overlaps A
        fkf.fkf_gemm_f64(ctx, A, B, A)
    assert e.value.status == fkf.FKF_EINVAL
    with pytest.raises(fkf.FkfError):  # leading dimension below the row length
        fkf._check(fkf._lib.fkf_gemm_f64(ctx.ptr, 0, 0, 8, 8, 8, 1.0, fkf._ptr(A), 4, fkf._ptr(B), 8, 0.0,
                                         fkf._ptr(torch.zeros((8, 8), dtype=torch.float64, device="cuda")), 8), ctx)
    C = torch.ones((8, 8), dtype=torch.float64, device="cuda")
    fkf.fkf_gemm_f64(ctx, A[:, :0], B[:0, :], C, beta=2.0)  # K = 0: C = beta C
    assert torch.equal(C, torch.full((8, 8), 2.0, dtype=torch.float64, device="cuda"))
    fkf.fkf_destroy(ctx)
