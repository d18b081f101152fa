"""H-matrix apply on the GPU (through the C-ABI) against the oracle's exact
Matern products (direct summation / dense Gamma)."""

import numpy as np
import pytest

import synth
from oracle import covariance
from tests.helpers import lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fkf():
    from paper_1405_2276_gb300 import build

    build()
    return lib()


@pytest.fixture(scope="module")
def ctx(fkf):
    c = fkf.fkf_create(0)
    yield c
    fkf.fkf_destroy(c)


def _apply(fkf, hm, X, prec):
    import torch

    dt = torch.float64 if prec == fkf.FKF_FP64 else torch.float32
    Xt = torch.from_numpy(X).to("cuda", dt).contiguous()
    Yt = torch.empty_like(Xt)
    fkf.fkf_hmatrix_apply(hm, Xt, Yt)
    return Yt.double().cpu().numpy()


CASES = [
    # grid, leaf, nu, ell, precision, aca_tol, tolerance on max|err|/max|ref|
    ((37, 23), 16, 1.5, 0.2, 0, 1e-10, 2e-8),
    ((32, 32), 64, 1.5, 0.2, 0, 1e-10, 2e-8),
    ((64, 48), 32, 0.5, 0.1, 0, 1e-10, 2e-8),
    ((37, 23), 16, 1.5, 0.2, 1, 1e-10, 2e-5),
    ((64, 48), 32, 0.5, 0.1, 1, 1e-8, 2e-5),
]


@pytest.mark.parametrize("grid,leaf,nu,ell,prec,tol,bound", CASES)
def test_apply_matches_dense_gamma(fkf, ctx, grid, leaf, nu, ell, prec, tol, bound):
    pts = synth.grid_points_2d(*grid)
    n = pts.shape[0]
    G = covariance.dense_gamma(pts, nu, ell, 1.0)
    hm = fkf.fkf_hmatrix_build(ctx, pts, nu, ell, 1.0, leaf=leaf, eta=1.0, aca_tol=tol, k_cap=64, precision=prec)
    info = fkf.fkf_hmatrix_info(hm)
    assert info["n"] == n and info["n_far"] > 0
    rng = np.random.default_rng(7)
    for ncols in (1, 7, 130, 300):
        X = rng.standard_normal((n, ncols))
        Y = _apply(fkf, hm, X, prec)
        ref = G @ X
        err = np.abs(Y - ref).max() / np.abs(ref).max()
        assert err < bound, (ncols, err)
    fkf.fkf_hmatrix_destroy(hm)


@pytest.mark.parametrize("prec", [0, 1])
def test_eta_zero_is_exact_and_symmetric(fkf, ctx, prec):
    """eta = 0: every block dense, so Gamma_H = Gamma up to rounding; the
    densified operator is exactly symmetric (each entry is stored once)."""
    pts = synth.grid_points_2d(20, 13)
    n = pts.shape[0]
    G = covariance.dense_gamma(pts, 1.5, 0.3, 2.0)
    hm = fkf.fkf_hmatrix_build(ctx, pts, 1.5, 0.3, 2.0, leaf=16, eta=0.0, precision=prec)
    assert fkf.fkf_hmatrix_info(hm)["n_far"] == 0
    D = fkf.fkf_hmatrix_densify(hm, n)
    np.testing.assert_array_equal(D, D.T)
    np.testing.assert_allclose(D, G, rtol=0, atol=(1e-15 if prec == 0 else 1e-7) * 2.0)
    fkf.fkf_hmatrix_destroy(hm)


def test_compressed_operator_exactly_symmetric(fkf, ctx):
    pts = synth.grid_points_2d(40, 30)
    n = pts.shape[0]
    G = covariance.dense_gamma(pts, 0.5, 0.1, 1.0)
    for prec, engine in ((0, 0), (1, 0), (1, 1), (1, 2)):
        hm = fkf.fkf_hmatrix_build(ctx, pts, 0.5, 0.1, 1.0, leaf=32, eta=1.0, aca_tol=1e-6, precision=prec)
        fkf.fkf_hmatrix_set_engine(hm, engine)
        D = fkf.fkf_hmatrix_densify(hm, n)
        if engine == 0:
            # SIMT engines multiply each stored entry the same way in both orientations
            np.testing.assert_array_equal(D, D.T)
        else:
            # tensor cores accumulate the 3xTF32 terms in their own order: symmetric to rounding
            assert np.abs(D - D.T).max() < 1e-6 * np.abs(D).max()
        # block-wise relative Frobenius tolerance 1e-6 -> global relative Frobenius error of that order
        assert np.linalg.norm(D - G) / np.linalg.norm(G) < 1e-5
        fkf.fkf_hmatrix_destroy(hm)


def test_permutation_is_a_permutation(fkf, ctx):
    pts = synth.grid_points_2d(37, 23)
    hm = fkf.fkf_hmatrix_build(ctx, pts, 1.5, 0.2, 1.0, leaf=16)
    p = fkf.fkf_hmatrix_permutation(hm, pts.shape[0])
    np.testing.assert_array_equal(np.sort(p), np.arange(pts.shape[0]))
    fkf.fkf_hmatrix_destroy(hm)


def test_ragged_3d_points(fkf, ctx):
    pts = synth.grid_points_3d(9, 7, 11)
    n = pts.shape[0]
    G = covariance.dense_gamma(pts, 0.5, 0.3, 1.0)
    hm = fkf.fkf_hmatrix_build(ctx, pts, 0.5, 0.3, 1.0, leaf=40, eta=1.0, aca_tol=1e-10, k_cap=48)
    X = np.random.default_rng(3).standard_normal((n, 33))
    Y = _apply(fkf, hm, X, 0)
    assert np.abs(Y - G @ X).max() / np.abs(G @ X).max() < 2e-8
    fkf.fkf_hmatrix_destroy(hm)


@pytest.mark.parametrize("prec,bound", [(0, 1e-6), (1, 3e-5)])
def test_medium_grid_sampled_rows(fkf, ctx, prec, bound):
    """256 x 256 grid (N = 65,536), nu = 3/2, ell = 0.1, leaf 64, ACA 1e-8,
    eta = 1, rank cap 32: sampled rows of Gamma_H X against direct sums."""
    pts = synth.grid_points_2d(256, 256)
    n = pts.shape[0]
    hm = fkf.fkf_hmatrix_build(ctx, pts, 1.5, 0.1, 1.0, leaf=64, eta=1.0, aca_tol=1e-8, k_cap=32, precision=prec)
    rng = np.random.default_rng(11)
    X = rng.standard_normal((n, 200))
    Y = _apply(fkf, hm, X, prec)
    rows = rng.choice(n, 48, replace=False)
    ref = covariance.gamma_rows_times(pts, rows, X, 1.5, 0.1, 1.0)
    err = np.abs(Y[rows] - ref).max() / np.abs(ref).max()
    assert err < bound, err
    fkf.fkf_hmatrix_destroy(hm)


def test_invalid_arguments(fkf, ctx):
    pts = synth.grid_points_2d(8, 8)
    with pytest.raises(fkf.FkfError) as e:
        fkf.fkf_hmatrix_build(ctx, pts, 0.7, 0.2, 1.0)
    assert e.value.status == fkf.FKF_EINVAL
    with pytest.raises(fkf.FkfError):
        fkf.fkf_hmatrix_build(ctx, pts, 0.5, -1.0, 1.0)
    hm = fkf.fkf_hmatrix_build(ctx, pts, 0.5, 0.2, 1.0, leaf=8)
    import torch

    X = torch.zeros((64, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(fkf.FkfError):  # X and Y overlap
        fkf.fkf_hmatrix_apply(hm, X, X)
    for engine in (1, 2):  # tensor-core engines need an FP32 operator
        with pytest.raises(fkf.FkfError):
            fkf.fkf_hmatrix_set_engine(hm, engine)
    with pytest.raises(fkf.FkfError):  # no engine 4
        fkf.fkf_hmatrix_set_engine(hm, 4)
    fkf.fkf_hmatrix_destroy(hm)


def test_engine_switch_round_trip(fkf, ctx):
    """Switching the tensor-core format rewrites the operator stream and
    clears the slot workspace: 1 -> 2 -> 1 -> 2 repeats each format's result
    bit for bit."""
    import torch

    pts = synth.grid_points_2d(96, 80)
    n = pts.shape[0]
    hm = fkf.fkf_hmatrix_build(ctx, pts, 1.5, 0.1, 1.0, leaf=32, eta=1.0, aca_tol=1e-8, k_cap=32, precision=1)
    X = torch.from_numpy(np.random.default_rng(21).standard_normal((n, 300))).to("cuda", torch.float32)
    out = {}
    for engine in (1, 2, 1, 2):
        fkf.fkf_hmatrix_set_engine(hm, engine)
        Y = torch.empty_like(X)
        fkf.fkf_hmatrix_apply_clustered(hm, X, Y)
        if engine in out:
            assert torch.equal(out[engine], Y), engine
        out[engine] = Y
    assert (out[1] - out[2]).abs().max().item() < 1e-5 * out[1].abs().max().item()
    fkf.fkf_hmatrix_destroy(hm)


@pytest.mark.parametrize("engine", [1, 2])
@pytest.mark.parametrize("grid,leaf,ncols", [((37, 23), 16, 300), ((64, 48), 32, 130), ((256, 256), 64, 260)])
def test_tensor_core_engine_matches_simt_and_dense(fkf, ctx, grid, leaf, ncols, engine):
    """The tcgen05 engines (1: 3xTF32, 2: scaled 2xFP16) against the FP64
    apply of the same H-matrix (same cluster tree, block tree and ACA
    pivots): the error must be of the FP32 SIMT engine's size (all accumulate
    in FP32), and against the exact product on small grids."""
    import torch

    pts = synth.grid_points_2d(*grid)
    n = pts.shape[0]
    hm = fkf.fkf_hmatrix_build(ctx, pts, 0.5, 0.1, 1.0, leaf=leaf, eta=1.0, aca_tol=1e-8, k_cap=32, precision=1)
    h64 = fkf.fkf_hmatrix_build(ctx, pts, 0.5, 0.1, 1.0, leaf=leaf, eta=1.0, aca_tol=1e-8, k_cap=32, precision=0)
    rng = np.random.default_rng(13)
    Xn = rng.standard_normal((n, ncols)).astype(np.float32).astype(np.float64)
    X = torch.from_numpy(Xn).to("cuda", torch.float32)
    Y_tc = torch.empty_like(X)
    Y_simt = torch.empty_like(X)
    fkf.fkf_hmatrix_set_engine(hm, engine)
    fkf.fkf_hmatrix_apply_clustered(hm, X, Y_tc)
    fkf.fkf_hmatrix_set_engine(hm, 0)
    fkf.fkf_hmatrix_apply_clustered(hm, X, Y_simt)
    X64 = torch.from_numpy(Xn).cuda()
    Y64 = torch.empty_like(X64)
    fkf.fkf_hmatrix_apply_clustered(h64, X64, Y64)
    a = Y_tc.double().cpu().numpy()
    b = Y_simt.double().cpu().numpy()
    c = Y64.cpu().numpy()
    assert np.isfinite(a).all()
    e_tc = np.abs(a - c).max() / np.abs(c).max()
    e_simt = np.abs(b - c).max() / np.abs(c).max()
    print(f"grid {grid} engine {engine}: tensor-core error {e_tc:.2e}, SIMT error {e_simt:.2e} (vs FP64 apply)")
    # 3xTF32 drops the lo*lo term (2^-22 relative per product) and accumulates in
    # the tensor core's FP32: FP32-level error, a small multiple of the SIMT engine's
    assert e_tc < max(10 * e_simt, 1e-5) and e_tc < 1e-4
    if n <= 4096:
        perm = fkf.fkf_hmatrix_permutation(hm, n)
        G = covariance.dense_gamma(pts[perm], 0.5, 0.1, 1.0)  # cluster order
        ref = G @ Xn
        assert np.abs(a - ref).max() / np.abs(ref).max() < 2e-5
    fkf.fkf_hmatrix_destroy(hm)
    fkf.fkf_hmatrix_destroy(h64)


def test_default_engine_as_built(fkf, ctx):
    """An FP32 operator starts on the scaled-FP16 tensor-core engine with the
    stream written at build time (no engine switch before the first apply)."""
    import torch

    pts = synth.grid_points_2d(48, 40)
    n = pts.shape[0]
    hm = fkf.fkf_hmatrix_build(ctx, pts, 1.5, 0.2, 1.0, leaf=32, eta=1.0, aca_tol=1e-8, k_cap=32, precision=1)
    assert fkf.fkf_hmatrix_get_engine(hm) == 2
    X = torch.from_numpy(np.random.default_rng(4).standard_normal((n, 40))).to("cuda", torch.float32)
    Y = torch.empty_like(X)
    fkf.fkf_hmatrix_apply_clustered(hm, X, Y)
    fkf.fkf_hmatrix_set_engine(hm, 0)
    Y0 = torch.empty_like(X)
    fkf.fkf_hmatrix_apply_clustered(hm, X, Y0)
    assert (Y - Y0).abs().max().item() < 2e-5 * Y0.abs().max().item()
    fkf.fkf_hmatrix_destroy(hm)


def test_autotune_keeps_results(fkf, ctx):
    """The autotuner picks a pipeline shape; both shapes give the same
    product bit for bit (the same MMAs in the same order per tile)."""
    import torch

    pts = synth.grid_points_2d(80, 72)
    n = pts.shape[0]
    hm = fkf.fkf_hmatrix_build(ctx, pts, 0.5, 0.1, 1.0, leaf=32, eta=1.0, aca_tol=1e-8, k_cap=32, precision=1)
    X = torch.from_numpy(np.random.default_rng(8).standard_normal((n, 300))).to("cuda", torch.float32)
    Y0 = torch.empty_like(X)
    fkf.fkf_hmatrix_apply_clustered(hm, X, Y0)
    v, ms = fkf.fkf_hmatrix_autotune(hm, 300)
    assert v in (0, 1) and ms > 0
    Y1 = torch.empty_like(X)
    fkf.fkf_hmatrix_apply_clustered(hm, X, Y1)
    assert torch.equal(Y0, Y1)
    fkf.fkf_hmatrix_set_engine(hm, 1)
    assert fkf.fkf_hmatrix_autotune(hm, 300) == (v, 0.0)  # nothing to tune on engine 1
    fkf.fkf_hmatrix_destroy(hm)


def test_release_values_keeps_tensor_core_results(fkf, ctx):
    """fkf_hmatrix_release_values frees the FP32 value copies: the tensor-core
    apply gives bitwise the same result, the paths that read the values refuse."""
    import torch

    pts = synth.grid_points_2d(48, 40)
    n = pts.shape[0]
    hm = fkf.fkf_hmatrix_build(ctx, pts, 1.5, 0.15, 1.0, leaf=32, eta=1.0, aca_tol=1e-8, precision=fkf.FKF_FP32)
    X = torch.from_numpy(np.random.default_rng(3).standard_normal((n, 70))).float().cuda()
    Y0 = torch.empty_like(X)
    fkf.fkf_hmatrix_apply(hm, X, Y0)
    before = fkf.fkf_hmatrix_info(hm)["device_bytes"]  # the apply's workspaces included
    fkf.fkf_hmatrix_release_values(hm)
    assert fkf.fkf_hmatrix_info(hm)["device_bytes"] < before
    Y1 = torch.empty_like(X)
    fkf.fkf_hmatrix_apply(hm, X, Y1)
    assert torch.equal(Y0, Y1)
    for call in (lambda: fkf.fkf_hmatrix_set_engine(hm, 0),
                 lambda: fkf.fkf_hmatrix_apply_clustered_noalloc(hm, X, Y1)):
        with pytest.raises(fkf.FkfError) as e:
            call()
        assert e.value.status == fkf.FKF_ESTATE
    fkf.fkf_hmatrix_destroy(hm)
    h64 = fkf.fkf_hmatrix_build(ctx, pts, 1.5, 0.15, 1.0, leaf=32, precision=fkf.FKF_FP64)
    with pytest.raises(fkf.FkfError):
        fkf.fkf_hmatrix_release_values(h64)
    fkf.fkf_hmatrix_destroy(h64)
