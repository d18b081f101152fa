"""The FP32 filter step hands H^T to the tensor-core H-apply as its sparse
column index (the FP16 split engine scatters the entries straight into its
split format, clearing the previous step's entries) instead of a dense H^T.
Both routes must give the same filter, bit for bit: FKF_STEP_DENSE_HT forces
the dense route on a second, identically built operator.  The operator
sequence changes the ray set (entries to clear), repeats it (kept basis) and
carries repeated column indices in a row (summed in order)."""

import numpy as np
import pytest

import synth
from tests.helpers import lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fkf():
    from paper_1405_2276_gb300 import build

    build()
    return lib()


def _with_repeats(h, rng):
    """The same operator with some entries split in two (same column, values
    0.25 v and 0.75 v next to each other)."""
    rp, col, val = [0], [], []
    for j in range(h.nrows):
        a, b = int(h.rowptr[j]), int(h.rowptr[j + 1])
        for p in range(a, b):
            if rng.random() < 0.2:
                col += [h.col[p], h.col[p]]
                val += [0.25 * h.val[p], 0.75 * h.val[p]]
            else:
                col.append(h.col[p])
                val.append(h.val[p])
        rp.append(len(col))
    return synth.Csr(np.asarray(rp, np.int64), np.asarray(col, np.int32), np.asarray(val, np.float64),
                     h.ncols)


def test_sparse_and_dense_ht_give_identical_filters(fkf):
    rng = np.random.default_rng(synth.BASE_SEED + 31)
    nx = ny = 72
    pts = synth.grid_points_2d(nx, ny)
    p0, p1 = synth.cross_well_geometry_2d(8, 8)
    Ha = synth.trace_rays_2d(nx, ny, p0, p1)
    Hb, Hc = synth.varying_ray_operators(rng, nx, ny, [50, 90])
    Hd = _with_repeats(Hb, rng)
    seq = [Ha, Ha, Hb, Hc, Hd, Hd, Ha]
    ys = [rng.standard_normal(h.nrows) * 0.3 for h in seq]
    n = pts.shape[0]
    ctx = fkf.fkf_create(0)
    runs = []
    for flags in (0, fkf.FKF_STEP_DENSE_HT):
        hm = fkf.fkf_hmatrix_build(ctx, pts, 1.5, 0.15, 1.0, leaf=64, eta=1.0, precision=fkf.FKF_FP32)
        assert fkf.fkf_hmatrix_get_engine(hm) == 2
        f = fkf.fkf_filter_create(hm, None, 0.0, 1e-12, 90, 400)
        nlls, paths = [], []
        for k, h in enumerate(seq):
            nlls.append(fkf.fkf_filter_step(f, ys[k], h.nrows, h.rowptr, h.col, h.val, None, 1e-4, flags=flags))
            paths.append(fkf.fkf_filter_get_stats(f)["last_path"])
        st = fkf.fkf_filter_get(f, n)
        runs.append((nlls, paths, st["s"].copy(), st["D"].copy(), st["r"]))
        fkf.fkf_filter_destroy(f)
        fkf.fkf_hmatrix_destroy(hm)
    fkf.fkf_destroy(ctx)
    (n0, p0_, s0, d0, r0), (n1, p1_, s1, d1, r1) = runs
    assert p0_ == p1_ and 1 in p0_ and 0 in p0_[1:]  # kept and merge steps both ran
    assert r0 == r1
    assert n0 == n1
    assert np.array_equal(s0, s1)
    assert np.array_equal(d0, d1)
