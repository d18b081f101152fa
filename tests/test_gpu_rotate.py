"""Tensor-core rotation product C = A E (the W' = [W G] E of the merge step)
through the C-ABI, against the FP64 product of the same FP32 inputs."""

import numpy as np
import pytest

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


def _bound(A, E):
    # 3xTF32 keeps each product to ~2^-21 relative; the tensor core adds each
    # MMA's K = 8 products into the FP32 accumulator with one rounding (not
    # IEEE per-addition), whose error grows about linearly with K (measured:
    # 2.6e-6 of sum_k |A_ik E_kj| at K = 2048).  1e-5 of that sum covers
    # K <= 4096 and is far below what a wrong element or index gives.
    return 1e-5 * (np.abs(A) @ np.abs(E)).max() + 1e-30


# rows, K, ncols, lda pad, column offset of A (unaligned start), lde pad, ldc pad
CASES = [
    (1000, 37, 300, 3, 1, 5, 2),
    (384, 16, 256, 0, 0, 0, 0),
    (4097, 300, 513, 0, 2, 0, 7),
    (130, 1, 1, 0, 0, 0, 0),
    (2048, 2048, 1024, 0, 0, 0, 0),
]


@pytest.mark.parametrize("rows,K,ncols,pa,off,pe,pc", CASES)
def test_rotate_matches_fp64_product(fkf, ctx, rows, K, ncols, pa, off, pe, pc):
    import torch

    rng = np.random.default_rng(rows + 7 * K + ncols)
    Abig = rng.standard_normal((rows, off + K + pa)).astype(np.float32)
    Ebig = rng.standard_normal((K + 3, ncols + pe)).astype(np.float32)
    A_d = torch.from_numpy(Abig).cuda()[:, off:off + K]
    E_d = torch.from_numpy(Ebig).cuda()
    C_d = torch.full((rows, ncols + pc), float("nan"), dtype=torch.float32, device="cuda")
    fkf.fkf_rotate_f32(ctx, A_d, E_d, C_d, K=K, ncols=ncols)
    A = Abig[:, off:off + K].astype(np.float64)
    E = Ebig[:K, :ncols].astype(np.float64)
    ref = A @ E
    got = C_d.cpu().numpy().astype(np.float64)
    assert np.isfinite(got[:, :ncols]).all()
    assert np.isnan(got[:, ncols:]).all()  # columns past ncols untouched
    err = np.abs(got[:, :ncols] - ref).max()
    print(f"rotate {rows}x{K}x{ncols}: max err {err:.2e}, bound {_bound(A, E):.2e}")
    assert err <= _bound(A, E), err


def test_rotate_k_zero_gives_zero(fkf, ctx):
    import torch

    A = torch.ones((200, 4), dtype=torch.float32, device="cuda")
    E = torch.ones((4, 40), dtype=torch.float32, device="cuda")
    C = torch.full((200, 40), 5.0, dtype=torch.float32, device="cuda")
    fkf.fkf_rotate_f32(ctx, A, E, C, K=0)
    assert (C == 0).all()


def test_rotate_full_size_sampled_rows(fkf, ctx):
    """The merge step's size: N = 262,144 rows, K = r + m = 2048, 1024 columns
    (rows sampled against FP64 sums)."""
    import torch

    n, K, nc = 262144, 2048, 1024
    g = torch.Generator(device="cuda").manual_seed(5)
    A = torch.randn((n, K), generator=g, device="cuda", dtype=torch.float32)
    E = torch.randn((K, nc), generator=g, device="cuda", dtype=torch.float32) / 32
    C = torch.empty((n, nc), dtype=torch.float32, device="cuda")
    fkf.fkf_rotate_f32(ctx, A, E, C)
    rows = np.random.default_rng(3).choice(n, 64, replace=False)
    An = A[rows].cpu().numpy().astype(np.float64)
    En = E.cpu().numpy().astype(np.float64)
    ref = An @ En
    err = np.abs(C[rows].cpu().numpy() - ref).max()
    assert err <= _bound(An, En), err


def test_rotate_rejects_bad_arguments(fkf, ctx):
    import torch

    A = torch.zeros((64, 8), dtype=torch.float32, device="cuda")
    E = torch.zeros((8, 16), dtype=torch.float32, device="cuda")
    C = torch.zeros((64, 16), dtype=torch.float32, device="cuda")
    with pytest.raises(fkf.FkfError):  # K > rows of E
        fkf.fkf_rotate_f32(ctx, A, E[:4], C, K=8)
    with pytest.raises(fkf.FkfError):  # C overlaps A
        fkf.fkf_rotate_f32(ctx, A, E, A[:, :4].as_strided((64, 4), (8, 1)), K=8)
