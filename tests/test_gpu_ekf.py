"""Extended filter with the Box-Cox measurement map (Sec. 4.2, Alg. extkalman)
on the GPU, through fkf_filter_step_ekf, against the dense extended filter of
the oracle (O1e).

The measurements are y_k = H s(x_k) + v_k with s(x) = ((x + a)/a)^a (Eq.
nonlinear), x_k a random walk of the transformed field.  The Jacobian
H_k = H diag(s'(x_pred)) changes every step, so every step runs the general
path (GEP, orthonormalisation, merge, rotation) and the rank grows until the
truncation bounds it.  FP64 path: relative 1e-10 with no truncation (the 1e-12 rounding floor of trunc_tol), relative 1e-9: a Jacobian that changes by a
rescaling of H's columns brings new directions whose Gamma^-1-norm outside
span(W) is small, and the orthonormalisation's rank-revealing threshold
(1e-10, which keeps X^T W = I to working precision) drops information of that
relative size (observed 1e-10 to 4e-10); and against O1e with the same
truncation at the paper's tolerance 1e-5.
"""

import numpy as np
import pytest

import synth
from oracle import covariance, kalman
from tests.helpers import lib, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fkf():
    from paper_1405_2276_gb300 import build

    build()
    return lib()


def _problem(a, steps=6, nx=24, ny=20, src=6, rec=5, sigma2=0.05, ell=0.25, noise=1e-4, seed=301):
    rng = np.random.default_rng(synth.BASE_SEED + seed)
    pts = synth.grid_points_2d(nx, ny)
    p0, p1 = synth.cross_well_geometry_2d(src, rec)
    H = synth.trace_rays_2d(nx, ny, p0, p1)
    truth = synth.random_walk_truth(rng, (nx, ny), steps, ell, sigma2)
    Hd = synth.csr_to_dense(H)
    ys = [Hd @ kalman.boxcox_state(truth[k], a) + np.sqrt(noise) * rng.standard_normal(H.nrows)
          for k in range(steps)]
    G = covariance.dense_gamma(pts, 1.5, ell, sigma2)
    return pts, H, Hd, ys, G, (1.5, ell, sigma2), noise


def _run(fkf, pts, H, ys, kern, noise, a, trunc_tol, r_max, precision=0):
    import torch

    n = pts.shape[0]
    ctx = fkf.fkf_create(0)
    hm = fkf.fkf_hmatrix_build(ctx, pts, *kern, leaf=32, eta=0.0, precision=precision)
    f = fkf.fkf_filter_create(hm, None, 0.0, trunc_tol, H.nrows, r_max)
    out = []
    for y in ys:
        nll = fkf.fkf_filter_step_ekf(f, y, H.nrows, H.rowptr, H.col, H.val, a, None, noise)
        st = fkf.fkf_filter_get(f, n)
        v = torch.empty(n, dtype=torch.float64, device="cuda")
        fkf.fkf_variance(f, v)
        W = torch.empty((n, max(st["r"], 1)), dtype=torch.float64 if precision == 0 else torch.float32,
                        device="cuda")
        fkf.fkf_filter_get(f, n, want_s=False, want_D=False, W=W)
        out.append(dict(s=st["s"], D=st["D"], r=st["r"], alpha=st["alpha"], nll=nll, var=v.cpu().numpy(),
                        W=W.double().cpu().numpy()[:, : st["r"]],
                        path=fkf.fkf_filter_get_stats(f)["last_path"]))
    orth = fkf.fkf_filter_orthonormality(f)
    fkf.fkf_filter_destroy(f)
    fkf.fkf_hmatrix_destroy(hm)
    fkf.fkf_destroy(ctx)
    return out, orth


@pytest.mark.parametrize("a", [2.0, 4.0, 6.0])
def test_ekf_matches_dense_extended_filter(fkf, a):
    pts, H, Hd, ys, G, kern, noise = _problem(a)
    ref = kalman.ekf_dense(G, [(y, Hd, noise) for y in ys], a)
    got, orth = _run(fkf, pts, H, ys, kern, noise, a, 1e-12, H.nrows * len(ys))
    worst = 0.0
    for k, (g, b) in enumerate(zip(got, ref)):
        Sig = g["alpha"] * G - (g["W"] * g["D"]) @ g["W"].T
        parts = (rel_err(g["s"], b["s"]), rel_err(g["var"], b["var"]), rel_err(Sig, b["Sigma"]),
                 abs(g["nll"] - b["nll"]) / abs(b["nll"]))
        e = max(parts)
        worst = max(worst, e)
        assert e < 1e-9, (k, parts)
        assert g["path"] == 0  # a new Jacobian every step: the merge path
    assert got[-1]["r"] > H.nrows  # the rank grew past one step's measurements
    # directions accepted just above the orthonormalisation's threshold tau_o = 1e-10 carry a
    # Gamma^-1-orthonormality error of order eps / tau_o (observed 2e-7 to 3e-7)
    print(f"EKF a={a:g}: orthonormality {orth:.1e}")
    assert orth < 1e-5
    print(f"EKF a={a:g}: worst rel err vs O1e {worst:.2e}, ranks {[g['r'] for g in got]}")


def test_ekf_truncated_at_paper_tolerance(fkf):
    """trunc_tol = 1e-5 (the paper's EKF setting): the GPU's ranks and results
    against O1e with the same truncation after every update."""
    a = 4.0
    pts, H, Hd, ys, G, kern, noise = _problem(a, steps=8, seed=302)
    ref = kalman.ekf_dense(G, [(y, Hd, noise) for y in ys], a, trunc_tol=1e-5)
    got, orth = _run(fkf, pts, H, ys, kern, noise, a, 1e-5, H.nrows * len(ys))
    ranks = [g["r"] for g in got]
    assert ranks == [q["r"] for q in ref]
    worst = 0.0
    for k, (g, b) in enumerate(zip(got, ref)):
        Sig = g["alpha"] * G - (g["W"] * g["D"]) @ g["W"].T
        e = max(rel_err(g["s"], b["s"]), rel_err(g["var"], b["var"]), rel_err(Sig, b["Sigma"]))
        worst = max(worst, e)
        assert e < 1e-9, (k, e)
    # against the untruncated extended filter: the truncation's own effect
    full = kalman.ekf_dense(G, [(y, Hd, noise) for y in ys], a)
    eff = max(rel_err(g["s"], b["s"]) for g, b in zip(got, full))
    print(f"EKF a=4 trunc 1e-5: ranks {ranks} (untruncated sum {H.nrows * len(ys)}), worst vs O1e(1e-5) "
          f"{worst:.2e}, s_hat vs untruncated {eff:.2e}")
    assert ranks[-1] < H.nrows * len(ys)


def test_ekf_with_unit_parameter_is_the_linear_step(fkf):
    """a = 1: s(x) = x + 1, so the extended step equals the linear step on the
    measurements y - H 1, bit for bit in the data-space algebra up to the
    innovation's summation order."""
    pts, H, Hd, ys, G, kern, noise = _problem(1.0, steps=4, seed=303)
    got, _ = _run(fkf, pts, H, ys, kern, noise, 1.0, 1e-12, H.nrows * 4)
    ref = kalman.kf_dense(G, [(y - Hd @ np.ones(pts.shape[0]), Hd, noise) for y in ys])
    for g, b in zip(got, ref):
        assert rel_err(g["s"], b["s"]) < 1e-10
        assert rel_err(g["var"], b["var"]) < 1e-10
