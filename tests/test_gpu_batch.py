"""Batched steps of independent filters with uneven sizes (fkf_filter_step_batched)
against the same filters stepped one at a time (bitwise), and every member of
the batch against the dense oracle: the FP64 members against O1 run on their
own compressed covariance Gamma_H (exported densely) at 1e-10, the FP32
members against O1 with the exact Matern covariance at 2e-4."""

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


SPECS = [  # grid, n_src, n_rec, nu, ell, precision
    ((16, 16), 4, 3, 0.5, 0.25, 0),
    ((24, 20), 5, 5, 1.5, 0.1, 0),
    ((32, 32), 8, 4, 1.5, 0.2, 1),
    ((20, 28), 3, 7, 0.5, 0.05, 1),
    ((40, 24), 6, 6, 1.5, 0.3, 0),
    ((12, 36), 2, 9, 0.5, 0.15, 1),
]


def _make(fkf, specs, steps):
    out = []
    for i, (grid, ns, nr, nu, ell, prec) in enumerate(specs):
        wl = synth.tomography_workload(grid, ns, nr, steps, ell, 1.0, 1e-4, seed=synth.BASE_SEED + 1000 * 3 + i)
        ctx = fkf.fkf_create(0)
        hm = fkf.fkf_hmatrix_build(ctx, wl["points"], nu, ell, 1.0, leaf=32, eta=1.0, aca_tol=1e-8, precision=prec)
        m = wl["H"].nrows
        f = fkf.fkf_filter_create(hm, None, 0.0, 1e-12, m, 2 * m)
        out.append(dict(wl=wl, ctx=ctx, hm=hm, f=f, spec=(grid, ns, nr, nu, ell, prec)))
    return out


def _free(fkf, objs):
    for o in objs:
        fkf.fkf_filter_destroy(o["f"])
        fkf.fkf_hmatrix_destroy(o["hm"])
        fkf.fkf_destroy(o["ctx"])


def test_batched_equals_sequential(fkf):
    steps = 3
    a = _make(fkf, SPECS, steps)
    b = _make(fkf, SPECS, steps)
    for k in range(steps):
        entries = []
        for o in a:
            h = o["wl"]["H"]
            entries.append((o["f"], o["wl"]["y"][k], h.rowptr, h.col, h.val, None, 1e-4))
        nll_b = fkf.fkf_filter_step_batched(entries)
        nll_s = []
        for o in b:
            h = o["wl"]["H"]
            nll_s.append(fkf.fkf_filter_step(o["f"], o["wl"]["y"][k], h.nrows, h.rowptr, h.col, h.val, None, 1e-4))
        assert nll_b == nll_s
    for oa, ob in zip(a, b):
        n = oa["wl"]["points"].shape[0]
        sa, sb = fkf.fkf_filter_get(oa["f"], n), fkf.fkf_filter_get(ob["f"], n)
        np.testing.assert_array_equal(sa["s"], sb["s"])
        np.testing.assert_array_equal(sa["D"], sb["D"])
    # every member against the dense oracle
    import torch

    for o in a:
        grid, ns, nr, nu, ell, prec = o["spec"]
        pts = o["wl"]["points"]
        n = pts.shape[0]
        G = fkf.fkf_hmatrix_densify(o["hm"], n) if prec == 0 else covariance.dense_gamma(pts, nu, ell, 1.0)
        Hd = synth.csr_to_dense(o["wl"]["H"])
        ref = kalman.kf_dense(G, [(o["wl"]["y"][k], Hd, 1e-4) for k in range(steps)], keep_cov=False)
        st = fkf.fkf_filter_get(o["f"], n)
        v = torch.empty(n, dtype=torch.float64, device="cuda")
        fkf.fkf_variance(o["f"], v)
        bound = 1e-10 if prec == 0 else 2e-4
        es, ev = rel_err(st["s"], ref[-1]["s"]), rel_err(v.cpu().numpy(), ref[-1]["var"])
        assert es < bound and ev < bound, (o["spec"], es, ev)
    _free(fkf, a)
    _free(fkf, b)


def test_batched_rejects_shared_context_and_reports_per_filter_status(fkf):
    objs = _make(fkf, SPECS[:2], 1)
    ctx = objs[0]["ctx"]
    f2 = fkf.fkf_filter_create(objs[0]["hm"], None, 0.0, 1e-12, 16, 32)
    h = objs[0]["wl"]["H"]
    with pytest.raises(fkf.FkfError) as e:
        fkf.fkf_filter_step_batched([(objs[0]["f"], objs[0]["wl"]["y"][0], h.rowptr, h.col, h.val, None, 1e-4),
                                     (f2, objs[0]["wl"]["y"][0], h.rowptr, h.col, h.val, None, 1e-4)])
    assert e.value.status == fkf.FKF_EINVAL
    # a bad noise variance in the second entry fails only that entry
    h1 = objs[1]["wl"]["H"]
    with pytest.raises(fkf.FkfError) as e:
        fkf.fkf_filter_step_batched([(objs[0]["f"], objs[0]["wl"]["y"][0], h.rowptr, h.col, h.val, None, 1e-4),
                                     (objs[1]["f"], objs[1]["wl"]["y"][0], h1.rowptr, h1.col, h1.val, None, -1.0)])
    assert e.value.status == fkf.FKF_EINVAL
    assert fkf.fkf_filter_get(objs[0]["f"], objs[0]["wl"]["points"].shape[0])["alpha"] == 1.0
    assert fkf.fkf_filter_get(objs[1]["f"], objs[1]["wl"]["points"].shape[0])["alpha"] == 0.0
    fkf.fkf_filter_destroy(f2)
    del ctx
    _free(fkf, objs)


SPECS32 = [  # uneven FP32 filters: grid, n_src, n_rec, nu, ell
    ((24, 24), 3, 4, 0.5, 0.1),
    ((64, 48), 8, 8, 1.5, 0.2),
    ((40, 40), 6, 10, 0.5, 0.05),
    ((96, 80), 12, 10, 1.5, 0.08),
    ((32, 56), 4, 6, 0.5, 0.3),
    ((72, 72), 10, 12, 1.5, 0.12),
]


def _make32(fkf, steps, engine=None):
    out = []
    for i, (grid, ns, nr, nu, ell) in enumerate(SPECS32):
        wl = synth.tomography_workload(grid, ns, nr, steps, ell, 1.0, 1e-4, seed=synth.BASE_SEED + 1000 * 4 + i)
        ctx = fkf.fkf_create(0)
        hm = fkf.fkf_hmatrix_build(ctx, wl["points"], nu, ell, 1.0, leaf=32, eta=1.0, aca_tol=1e-8, precision=1)
        if engine is not None and i == 1:
            fkf.fkf_hmatrix_set_engine(hm, engine)
        m = wl["H"].nrows
        f = fkf.fkf_filter_create(hm, None, 0.0, 1e-12, m, 2 * m)
        out.append(dict(wl=wl, ctx=ctx, hm=hm, f=f))
    return out


@pytest.mark.parametrize("engine", [None, 1])
def test_fp32_batch_merged_apply_bitwise(fkf, engine):
    """FP32 filters of uneven N and m: with one tensor-core format the batch's
    H-applies run as one merged launch per phase (engine None: all on the
    default engine); a filter on another format (engine 1) runs alone and the
    others stay merged.  Either way every result equals stepping the filters
    alone, bit for bit."""
    steps = 3
    a = _make32(fkf, steps, engine)
    b = _make32(fkf, steps, engine)
    for k in range(steps):
        entries = []
        for o in a:
            h = o["wl"]["H"]
            entries.append((o["f"], o["wl"]["y"][k], h.rowptr, h.col, h.val, None, 1e-4))
        nll_b, merged = fkf.fkf_filter_step_batched(entries, return_merged=True)
        assert merged == [engine is None or i != 1 for i in range(len(a))]
        nll_s = []
        for o in b:
            h = o["wl"]["H"]
            nll_s.append(fkf.fkf_filter_step(o["f"], o["wl"]["y"][k], h.nrows, h.rowptr, h.col, h.val, None, 1e-4))
        assert nll_b == nll_s
    for oa, ob in zip(a, b):
        n = oa["wl"]["points"].shape[0]
        sa, sb = fkf.fkf_filter_get(oa["f"], n), fkf.fkf_filter_get(ob["f"], n)
        np.testing.assert_array_equal(sa["s"], sb["s"])
        np.testing.assert_array_equal(sa["D"], sb["D"])
    _free(fkf, a)
    _free(fkf, b)
