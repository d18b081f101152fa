"""Adjoints on the GPU: the H-apply autograd op and the fixed-H filter NLL
gradient, against the oracle's batch-Gaussian gradients and central finite
differences (FP64 path)."""

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


@pytest.fixture(scope="module")
def ctx(fkf):
    c = fkf.fkf_create(0)
    yield c
    fkf.fkf_destroy(c)


def _problem(K=5):
    wl = workload(TINY, K)
    return wl, wl["points"], wl["H"]


def test_nll_matches_filter_steps(fkf, ctx):
    """The data-space NLL equals the general-path filter's per-step NLLs."""
    wl, pts, h = _problem(6)
    n, m = pts.shape[0], h.nrows
    rng = np.random.default_rng(2)
    s0 = rng.standard_normal(n) * 0.1
    alpha0 = 0.5
    hm = fkf.fkf_hmatrix_build(ctx, pts, *[TINY[k] for k in ("nu", "ell", "sigma2")], leaf=64, eta=0.0)
    f = fkf.fkf_filter_create(hm, s0, alpha0, 1e-12, m, 2 * m)
    total = sum(fkf.fkf_filter_step(f, wl["y"][k], m, h.rowptr, h.col, h.val, None, TINY["noise"]) for k in range(6))
    nll, *_ = fkf.fkf_nll_gradient(hm, wl["y"], h.rowptr, h.col, h.val, TINY["noise"], s0, alpha0, want_grads=False)
    assert abs(nll - total) < 1e-10 * abs(total)
    fkf.fkf_filter_destroy(f)
    fkf.fkf_hmatrix_destroy(hm)


@pytest.mark.parametrize("alpha0", [0.0, 0.7])
def test_gradients_match_oracle(fkf, ctx, alpha0):
    wl, pts, h = _problem(5)
    n, m = pts.shape[0], h.nrows
    sigma2, rho = 1.3, 2e-4
    rng = np.random.default_rng(3)
    s0 = rng.standard_normal(n) * 0.1
    hm = fkf.fkf_hmatrix_build(ctx, pts, TINY["nu"], TINY["ell"], sigma2, leaf=64, eta=0.0)
    nll, gy, gs0, gsig, grho = fkf.fkf_nll_gradient(hm, wl["y"], h.rowptr, h.col, h.val, rho, s0, alpha0)
    G1 = covariance.dense_gamma(pts, TINY["nu"], TINY["ell"], 1.0)
    Hd = synth.csr_to_dense(h)
    rnll, rgy, rgs0, rgsig, rgrho = kalman.nll_batch_and_gradients(G1, sigma2, rho, [Hd] * 5, list(wl["y"]), s0, alpha0)
    assert abs(nll - rnll) < 1e-10 * abs(rnll)
    assert rel_err(gy, np.stack(rgy)) < 1e-8
    assert rel_err(gs0, rgs0) < 1e-8
    assert abs(gsig - rgsig) < 1e-8 * max(1.0, abs(rgsig))
    assert abs(grho - rgrho) < 1e-8 * max(1.0, abs(rgrho))
    fkf.fkf_hmatrix_destroy(hm)


def test_gradients_match_central_differences(fkf, ctx):
    """Central differences of the library's own NLL (compressed Gamma_H)."""
    wl, pts, h = _problem(4)
    n = pts.shape[0]
    kern = (TINY["nu"], TINY["ell"])
    sigma2, rho = 1.0, 1e-4
    y = wl["y"].copy()

    def nll_at(sig, r, yy, s0):
        hm = fkf.fkf_hmatrix_build(ctx, pts, kern[0], kern[1], sig, leaf=64, eta=1.0, aca_tol=1e-10)
        v, *_ = fkf.fkf_nll_gradient(hm, yy, h.rowptr, h.col, h.val, r, s0, 0.0, want_grads=False)
        fkf.fkf_hmatrix_destroy(hm)
        return v

    hm = fkf.fkf_hmatrix_build(ctx, pts, kern[0], kern[1], sigma2, leaf=64, eta=1.0, aca_tol=1e-10)
    s0 = np.zeros(n)
    _, gy, gs0, gsig, grho = fkf.fkf_nll_gradient(hm, y, h.rowptr, h.col, h.val, rho, s0, 0.0)
    fkf.fkf_hmatrix_destroy(hm)
    e = 1e-5
    fd = (nll_at(sigma2 * (1 + e), rho, y, s0) - nll_at(sigma2 * (1 - e), rho, y, s0)) / (2 * e * sigma2)
    assert abs(fd - gsig) < 1e-5 * max(1.0, abs(gsig))
    fd = (nll_at(sigma2, rho * (1 + e), y, s0) - nll_at(sigma2, rho * (1 - e), y, s0)) / (2 * e * rho)
    assert abs(fd - grho) < 1e-5 * max(1.0, abs(grho))
    for k, j in [(0, 3), (3, 17)]:
        yp, ym = y.copy(), y.copy()
        yp[k, j] += 1e-6
        ym[k, j] -= 1e-6
        fd = (nll_at(sigma2, rho, yp, s0) - nll_at(sigma2, rho, ym, s0)) / 2e-6
        assert abs(fd - gy[k, j]) < 1e-5 * max(1.0, abs(fd))
    i = int(h.col[h.rowptr[5]])  # a cell on ray 5
    sp, sm = s0.copy(), s0.copy()
    sp[i] += 1e-6
    sm[i] -= 1e-6
    fd = (nll_at(sigma2, rho, y, sp) - nll_at(sigma2, rho, y, sm)) / 2e-6
    assert abs(fd - gs0[i]) < 1e-5 * max(1.0, abs(fd))


def test_autograd_functions(fkf, ctx):
    import torch

    from paper_1405_2276_gb300.autograd import FilterNLL, HApply

    pts = synth.grid_points_2d(12, 10)
    n = pts.shape[0]
    hm = fkf.fkf_hmatrix_build(ctx, pts, 0.5, 0.3, 1.7, leaf=16, eta=1.0, aca_tol=1e-12, precision=0)
    X = torch.randn(n, 3, dtype=torch.float64, device="cuda", requires_grad=True)
    s2 = torch.tensor(1.7, dtype=torch.float64, requires_grad=True)
    assert torch.autograd.gradcheck(lambda x: HApply.apply(x, s2, hm), (X,), eps=1e-6, atol=1e-8)
    C = torch.randn(n, 3, dtype=torch.float64, device="cuda")
    L = torch.sum(HApply.apply(X, s2, hm) * C)
    L.backward()
    G = covariance.dense_gamma(pts, 0.5, 0.3, 1.7)
    gx = G @ C.cpu().numpy()
    assert rel_err(X.grad.cpu().numpy(), gx) < 1e-10
    ref_s2 = float(np.sum(C.cpu().numpy() * (G @ X.detach().cpu().numpy()))) / 1.7
    assert abs(s2.grad.item() - ref_s2) < 1e-9 * abs(ref_s2)
    fkf.fkf_hmatrix_destroy(hm)
    # FilterNLL end to end through torch.autograd
    wl, ptsT, h = _problem(3)
    hmT = fkf.fkf_hmatrix_build(ctx, ptsT, TINY["nu"], TINY["ell"], TINY["sigma2"], leaf=64, eta=0.0)
    y = torch.tensor(wl["y"], dtype=torch.float64, requires_grad=True)
    s0 = torch.zeros(ptsT.shape[0], dtype=torch.float64, requires_grad=True)
    sig = torch.tensor(TINY["sigma2"], dtype=torch.float64, requires_grad=True)
    rho = torch.tensor(TINY["noise"], dtype=torch.float64, requires_grad=True)
    out = 2.0 * FilterNLL.apply(y, s0, sig, rho, hmT, h, 0.0)
    out.backward()
    G1 = covariance.dense_gamma(ptsT, TINY["nu"], TINY["ell"], 1.0)
    Hd = synth.csr_to_dense(h)
    rnll, rgy, rgs0, rgsig, rgrho = kalman.nll_batch_and_gradients(G1, TINY["sigma2"], TINY["noise"], [Hd] * 3,
                                                                   list(wl["y"]))
    assert abs(out.item() - 2 * rnll) < 1e-9 * abs(rnll)
    assert rel_err(y.grad.numpy(), 2 * np.stack(rgy)) < 1e-8
    assert abs(rho.grad.item() - 2 * rgrho) < 1e-8 * abs(rgrho)
    assert abs(sig.grad.item() - 2 * rgsig) < 1e-8 * max(1.0, abs(rgsig))
    fkf.fkf_hmatrix_destroy(hmT)
