"""The randomized GHEP (App. B, Alg. randomizedghepuncert) inside the filter
step on the GPU, through fkf_filter_set_randomized_ghep, against the oracle's
filter that takes its measurement information from the oracle's randomized
GHEP with the same Gaussian sketch (FP64 path, 1e-8), and against the exact
filter O1 when the sketch spans the range of H^T R^-1 H (k + p = m)."""

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


def _problem(seed, ms, nx=24, ny=24):
    rng = np.random.default_rng(synth.BASE_SEED + seed)
    pts = synth.grid_points_2d(nx, ny)
    ops = synth.varying_ray_operators(rng, nx, ny, ms)
    truth = synth.random_walk_truth(rng, (nx, ny), len(ms), 0.2, 1.0)
    ys = [synth.measurements(rng, h, truth[k], 1e-4) for k, h in enumerate(ops)]
    return rng, pts, ops, ys


def _run(fkf, pts, ops, ys, k, p, Om, r_max):
    import torch

    n = pts.shape[0]
    ctx = fkf.fkf_create(0)
    hm = fkf.fkf_hmatrix_build(ctx, pts, 1.5, 0.25, 1.0, leaf=32, eta=0.0)
    f = fkf.fkf_filter_create(hm, None, 0.0, 1e-12, max(h.nrows for h in ops), r_max)
    fkf.fkf_filter_set_randomized_ghep(f, k, p, torch.from_numpy(np.ascontiguousarray(Om)).cuda())
    out = []
    for y, h in zip(ys, ops):
        nll = fkf.fkf_filter_step(f, y, h.nrows, h.rowptr, h.col, h.val, None, 1e-4,
                                  flags=fkf.FKF_STEP_FULL_UPDATE)
        gr = fkf.fkf_filter_get_stats(f)["gep_rank"]
        st = fkf.fkf_filter_get(f, n)
        W = torch.empty((n, st["r"]), dtype=torch.float64, device="cuda")
        fkf.fkf_filter_get(f, n, want_s=False, want_D=False, W=W)
        out.append(dict(s=st["s"], alpha=st["alpha"], D=st["D"], W=W.cpu().numpy(), nll=nll, gep_rank=gr))
    fkf.fkf_filter_destroy(f)
    fkf.fkf_hmatrix_destroy(hm)
    fkf.fkf_destroy(ctx)
    return out


def test_randomized_ghep_matches_oracle_randomized_filter(fkf):
    ms = [20, 24, 18, 22, 20]
    rng, pts, ops, ys = _problem(401, ms)
    n = pts.shape[0]
    k, p = 8, 4
    Om = rng.standard_normal((n, k + p))
    G = covariance.dense_gamma(pts, 1.5, 0.25, 1.0)
    so = [(ys[i], synth.csr_to_dense(ops[i]), 1e-4) for i in range(len(ms))]
    ref = kalman.kf_dense_randomized_ghep(G, so, Om, k)
    got = _run(fkf, pts, ops, ys, k, p, Om, k * len(ms))
    worst = 0.0
    for i, (a, b) in enumerate(zip(got, ref)):
        assert a["gep_rank"] == k
        Sig = a["alpha"] * G - (a["W"] * a["D"]) @ a["W"].T
        e = max(rel_err(a["s"], b["s"]), rel_err(Sig, b["Sigma"]), abs(a["nll"] - b["nll"]) / abs(b["nll"]))
        worst = max(worst, e)
        assert e < 1e-8, (i, e)
    exact = kalman.kf_dense(G, so)
    approx = max(rel_err(a["s"], b["s"]) for a, b in zip(got, exact))
    print(f"randomized GHEP k={k} p={p}: worst vs oracle {worst:.2e}; s_hat vs the exact filter {approx:.2e}")


def test_randomized_ghep_with_spanning_sketch_is_the_exact_filter(fkf):
    ms = [12, 12, 12, 12]
    rng, pts, ops, ys = _problem(402, ms)
    n = pts.shape[0]
    Om = rng.standard_normal((n, 12))
    G = covariance.dense_gamma(pts, 1.5, 0.25, 1.0)
    ref = kalman.kf_dense(G, [(ys[i], synth.csr_to_dense(ops[i]), 1e-4) for i in range(len(ms))])
    got = _run(fkf, pts, ops, ys, 12, 0, Om, sum(ms))
    for i, (a, b) in enumerate(zip(got, ref)):
        Sig = a["alpha"] * G - (a["W"] * a["D"]) @ a["W"].T
        assert rel_err(a["s"], b["s"]) < 1e-9, i
        assert rel_err(Sig, b["Sigma"]) < 1e-9, i
