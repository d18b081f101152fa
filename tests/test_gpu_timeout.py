"""The bounded-wait path of the tensor-core H-apply (failure detection without
a GPU fault).

Every mbarrier wait inside the persistent kernel (producer -> MMA -> epilogue
hand-offs) gives up after a poll limit, marks its CTA failed and unwinds: the
MMA thread waits for the MMAs it issued, the producer for the bulk copies it
issued (both with the full default limit), TMEM is freed, and the host reads
the error flag as FKF_ETIMEOUT.  The test lowers the limit to 0 polls, so the
first pipeline wait of every role gives up at once (no wait is ever left
running), checks the status, and checks that the operator and the filter are
still usable: the next applies and steps with the default limit are bitwise
those of a run that never timed out, and a step that timed out left the
filter state unchanged.
"""

import numpy as np
import pytest

from tests.helpers import TINY, lib, workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fkf():
    from paper_1405_2276_gb300 import build

    build()
    return lib()


def test_apply_timeout_is_reported_and_recoverable(fkf):
    import torch

    wl = workload(TINY, 3)
    pts = wl["points"]
    n = pts.shape[0]
    ctx = fkf.fkf_create(0)
    hm = fkf.fkf_hmatrix_build(ctx, pts, TINY["nu"], TINY["ell"], TINY["sigma2"], leaf=64, eta=1.0, aca_tol=1e-8,
                               precision=fkf.FKF_FP32)
    assert fkf.fkf_hmatrix_get_engine(hm) == 2
    X = torch.from_numpy(np.random.default_rng(5).standard_normal((n, 48))).float().cuda()
    Y0 = torch.empty_like(X)
    fkf.fkf_hmatrix_apply(hm, X, Y0)
    fkf.fkf_hmatrix_set_wait_limit(hm, 0)
    Yt = torch.zeros_like(X)
    with pytest.raises(fkf.FkfError) as e:
        fkf.fkf_hmatrix_apply(hm, X, Yt)
    assert e.value.status == fkf.FKF_ETIMEOUT
    fkf.fkf_hmatrix_set_wait_limit(hm, -1)
    for _ in range(2):
        Y1 = torch.empty_like(X)
        fkf.fkf_hmatrix_apply(hm, X, Y1)
        assert torch.equal(Y1, Y0)
    fkf.fkf_hmatrix_destroy(hm)
    fkf.fkf_destroy(ctx)


def test_fp64_slice_engine_timeout_is_reported_and_recoverable(fkf):
    """The same unwind in the FP64 tensor-core engine (engine 3)."""
    import torch

    wl = workload(TINY, 3)
    pts = wl["points"]
    n = pts.shape[0]
    ctx = fkf.fkf_create(0)
    hm = fkf.fkf_hmatrix_build(ctx, pts, TINY["nu"], TINY["ell"], TINY["sigma2"], leaf=64, eta=1.0, aca_tol=1e-8,
                               precision=fkf.FKF_FP64)
    fkf.fkf_hmatrix_set_engine(hm, 3)
    X = torch.from_numpy(np.random.default_rng(6).standard_normal((n, 40))).cuda()
    Y0 = torch.empty_like(X)
    fkf.fkf_hmatrix_apply(hm, X, Y0)
    fkf.fkf_hmatrix_set_wait_limit(hm, 0)
    Yt = torch.zeros_like(X)
    with pytest.raises(fkf.FkfError) as e:
        fkf.fkf_hmatrix_apply(hm, X, Yt)
    assert e.value.status == fkf.FKF_ETIMEOUT
    fkf.fkf_hmatrix_set_wait_limit(hm, -1)
    for _ in range(2):
        Y1 = torch.empty_like(X)
        fkf.fkf_hmatrix_apply(hm, X, Y1)
        assert torch.equal(Y1, Y0)
    fkf.fkf_hmatrix_destroy(hm)
    fkf.fkf_destroy(ctx)


def test_filter_step_timeout_leaves_state_unchanged(fkf):
    wl = workload(TINY, 4)
    pts, h = wl["points"], wl["H"]
    n, m = pts.shape[0], h.nrows

    def make():
        ctx = fkf.fkf_create(0)
        hm = fkf.fkf_hmatrix_build(ctx, pts, TINY["nu"], TINY["ell"], TINY["sigma2"], leaf=64, eta=1.0,
                                   aca_tol=1e-8, precision=fkf.FKF_FP32)
        return ctx, hm, fkf.fkf_filter_create(hm, None, 0.0, 1e-12, m, 2 * m)

    def step(f, k):
        return fkf.fkf_filter_step(f, wl["y"][k], m, h.rowptr, h.col, h.val, None, TINY["noise"])

    ctx_a, hm_a, fa = make()
    ctx_b, hm_b, fb = make()
    na = [step(fa, 0), step(fa, 1)]
    fkf.fkf_filter_get(fa, n)  # both filters observed at the same point (same canonical state)
    na += [step(fa, 2), step(fa, 3)]
    nb = [step(fb, 0), step(fb, 1)]
    before = fkf.fkf_filter_get(fb, n)
    fkf.fkf_hmatrix_set_wait_limit(hm_b, 0)
    with pytest.raises(fkf.FkfError) as e:
        step(fb, 2)
    assert e.value.status == fkf.FKF_ETIMEOUT
    after = fkf.fkf_filter_get(fb, n)
    np.testing.assert_array_equal(after["s"], before["s"])
    np.testing.assert_array_equal(after["D"], before["D"])
    assert after["alpha"] == before["alpha"] and after["r"] == before["r"]
    fkf.fkf_hmatrix_set_wait_limit(hm_b, -1)
    nb += [step(fb, 2), step(fb, 3)]
    assert nb == na
    np.testing.assert_array_equal(fkf.fkf_filter_get(fb, n)["s"], fkf.fkf_filter_get(fa, n)["s"])
    for ctx, hm, f in ((ctx_a, hm_a, fa), (ctx_b, hm_b, fb)):
        fkf.fkf_filter_destroy(f)
        fkf.fkf_hmatrix_destroy(hm)
        fkf.fkf_destroy(ctx)
