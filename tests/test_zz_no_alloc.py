"""The allocation-free H-apply (fkf_hmatrix_apply_clustered_noalloc).

Callers that cannot call cudaMalloc -- a real-time loop that must not block in
the allocator, or a process whose device memory belongs to another allocator
-- use this entry point; it keeps its workspace in a fixed static device array
instead.  These tests call it through the C-ABI binding and compare it with the
regular fkf_hmatrix_apply_clustered on the same inputs, twice in a row (the
static array keeps the previous call's contents, which must not leak into the
next result).  This file is named to be collected last.
"""

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


@pytest.mark.parametrize(
    "grid,leaf,prec,ncols,tol",
    [
        ((37, 23), 16, 0, 70, 1e-12),    # small operator: one panel
        ((37, 23), 16, 1, 300, 2e-5),  # FP32: the regular apply may run on the tensor cores
        ((256, 256), 64, 0, 40, 1e-12),  # 65,536 points: several panels of the static scratch
    ],
)
def test_noalloc_apply_matches_regular_apply(fkf, grid, leaf, prec, ncols, tol):
    import torch

    ctx = fkf.fkf_create(0)
    pts = synth.grid_points_2d(*grid)
    n = pts.shape[0]
    hm = fkf.fkf_hmatrix_build(ctx, pts, 1.5, 0.1, 1.0, leaf=leaf, eta=1.0, aca_tol=1e-8, k_cap=32, precision=prec)
    dt = torch.float64 if prec == 0 else torch.float32
    rng = np.random.default_rng(21)
    Y_ref = None
    for call in range(2):
        X = torch.from_numpy(rng.standard_normal((n, ncols))).to("cuda", dt)
        Y_ref = torch.empty_like(X)
        fkf.fkf_hmatrix_apply_clustered(hm, X, Y_ref)
        Y = torch.full_like(X, float("nan"))
        fkf.fkf_hmatrix_apply_clustered_noalloc(hm, X, Y)
        ref = Y_ref.double().cpu().numpy()
        got = Y.double().cpu().numpy()
        assert np.isfinite(got).all()
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err <= tol, (call, err)
    fkf.fkf_hmatrix_destroy(hm)
    fkf.fkf_destroy(ctx)
