"""The library's own FP64 symmetric eigensolver (Householder tridiagonalisation,
divide and conquer, back-transformation) through fkf_eigh, against numpy's
eigvalsh (the definition: the spectrum) and the defining identities
A X = X diag(w), X^T X = I, on ragged sizes up to 3072 and on spectra with
clusters, repeated eigenvalues, wide dynamic range and low rank."""

import time

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


def _solve(fkf, ctx, A, want=None):
    import torch

    n = A.shape[0]
    At = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.time()
    fkf.fkf_eigh(ctx, At, w, want)
    torch.cuda.synchronize()
    dt = time.time() - t0
    k = n if want is None else want
    return w.cpu().numpy(), At.cpu().numpy()[:k].T.copy(), dt


def _check(A, w, X, k, tol=1e-12):
    n = A.shape[0]
    ref = np.linalg.eigvalsh(A)
    scale = max(np.abs(ref).max(), 1e-300)
    ew = np.abs(w - ref).max() / scale
    lam = w[n - k:]
    res = np.abs(A @ X - X * lam).max() / scale if k else 0.0
    orth = np.abs(X.T @ X - np.eye(k)).max() if k else 0.0
    assert ew < tol * max(1.0, n / 64), ew
    assert res < tol * max(1.0, n / 64), res
    assert orth < tol * max(1.0, n / 64), orth
    return ew, res, orth


@pytest.mark.parametrize("n", [1, 2, 3, 17, 31, 32, 33, 64, 65, 100, 257, 1000, 1024, 2048, 3072])
def test_random_symmetric(fkf, ctx, n):
    rng = np.random.default_rng(1000 + n)
    B = rng.standard_normal((n, n))
    A = B + B.T
    w, X, dt = _solve(fkf, ctx, A)
    ew, res, orth = _check(A, w, X, n)
    print(f"n={n}: eigenvalues {ew:.1e}, residual {res:.1e}, orthogonality {orth:.1e}, {dt * 1e3:.1f} ms")


@pytest.mark.parametrize("kind", ["cluster", "repeated", "decay", "lowrank", "diagonal"])
@pytest.mark.parametrize("n", [300, 1024])
def test_structured_spectra(fkf, ctx, kind, n):
    rng = np.random.default_rng(7)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    if kind == "cluster":
        ev = np.concatenate([1.0 + 1e-12 * rng.standard_normal(n // 3), rng.uniform(-1, 3, n - n // 3)])
    elif kind == "repeated":
        ev = np.repeat([1.0, 2.0, 3.0], n // 3 + 1)[:n]
    elif kind == "decay":
        ev = 10.0 ** rng.uniform(-14, 2, n)
    elif kind == "lowrank":
        ev = np.zeros(n)
        ev[:10] = rng.uniform(1, 2, 10)
    else:
        ev = rng.uniform(-1, 1, n)
        Q = np.eye(n)
    A = (Q * ev) @ Q.T
    A = 0.5 * (A + A.T)
    w, X, dt = _solve(fkf, ctx, A)
    ew, res, orth = _check(A, w, X, n)
    print(f"{kind} n={n}: eigenvalues {ew:.1e}, residual {res:.1e}, orthogonality {orth:.1e}")


@pytest.mark.parametrize("n,want", [(257, 40), (1024, 1), (2048, 1024)])
def test_top_eigenvectors_only(fkf, ctx, n, want):
    rng = np.random.default_rng(11)
    B = rng.standard_normal((n, n))
    A = B @ B.T / n
    w, X, dt = _solve(fkf, ctx, A, want)
    _check(A, w, X, want)
