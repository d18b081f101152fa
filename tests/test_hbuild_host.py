"""Host logic of the H-matrix construction, checked on the CPU (no GPU).

The library builds Gamma_H on the host (csrc/hbuild.cpp: cluster tree by
median bisection, block tree with the admissibility min(diam t, diam s) <=
eta dist(t, s), ACA for the admissible blocks, dense near tiles).  The test
compiles a small harness (tests/hbuild_dump.cpp) against that source with the
host C++ compiler, runs it on seeded point sets and checks the result against
definitions and the oracle's Matern kernel:
  * the cluster order is a permutation; children split their parent's range;
    leaves hold at most `leaf` points; every box contains its points;
  * the blocks (t, s) and their mirrors (s, t) cover every matrix entry
    exactly once;
  * every low-rank block is admissible and within its rank cap, and matches the
    exact kernel block to the block-wise relative Frobenius tolerance (the
    ACA's stopping rule is a heuristic: the bound allows a factor of 10);
  * near tiles hold the exact kernel values.
"""

import os
import shutil
import subprocess

import numpy as np
import pytest

import synth
from oracle import covariance

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1405_2276_gb300", "csrc")


@pytest.fixture(scope="module")
def dump_tool(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("no host C++ compiler")
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    inc = os.path.join(cuda, "include")
    if not os.path.exists(os.path.join(inc, "cuda_runtime.h")):
        pytest.skip("CUDA headers not found")
    out = str(tmp_path_factory.mktemp("hbuild") / "hbuild_dump")
    subprocess.run([gxx, "-O2", "-std=c++17", "-pthread", f"-I{CSRC}", f"-I{inc}",
                    os.path.join(ROOT, "tests", "hbuild_dump.cpp"), os.path.join(CSRC, "hbuild.cpp"), "-o", out],
                   check=True, capture_output=True)
    return out


class _Reader:
    def __init__(self, raw):
        self.raw, self.p = raw, 0

    def ints(self, n):
        v = np.frombuffer(self.raw, dtype=np.int64, count=n, offset=self.p)
        self.p += 8 * n
        return v

    def doubles(self, n):
        v = np.frombuffer(self.raw, dtype=np.float64, count=n, offset=self.p)
        self.p += 8 * n
        return v


def _build(tool, tmp_path, pts, nu, ell, sigma2, leaf, eta, tol, kcap):
    n, dim = pts.shape
    pin, pout = tmp_path / "pts.bin", tmp_path / "h.bin"
    np.ascontiguousarray(pts, dtype=np.float64).tofile(pin)
    subprocess.run([tool, str(pin), str(n), str(dim), repr(nu), repr(ell), repr(sigma2), str(leaf), repr(eta),
                    repr(tol), str(kcap), str(pout)], check=True)
    r = _Reader(pout.read_bytes())
    perm = r.ints(n).copy()
    ncl = int(r.ints(1)[0])
    cl = []
    for _ in range(ncl):
        b, e, c0, c1 = (int(x) for x in r.ints(4))
        lo, hi = r.doubles(3).copy(), r.doubles(3).copy()
        cl.append(dict(b=b, e=e, ch=(c0, c1), lo=lo[:dim], hi=hi[:dim]))
    far = []
    for _ in range(int(r.ints(1)[0])):
        t, s, k = (int(x) for x in r.ints(3))
        nt, ns = cl[t]["e"] - cl[t]["b"], cl[s]["e"] - cl[s]["b"]
        U = r.doubles(k * nt).reshape(k, nt).T
        V = r.doubles(k * ns).reshape(k, ns).T
        far.append((t, s, k, U, V))
    nnear = int(r.ints(1)[0])
    near = [tuple(int(x) for x in r.ints(2)) for _ in range(nnear)]
    tiles = []
    for t, s in near:
        nt, ns = cl[t]["e"] - cl[t]["b"], cl[s]["e"] - cl[s]["b"]
        tiles.append(r.doubles(nt * ns).reshape(nt, ns))
    assert r.p == len(r.raw)
    return perm, cl, far, near, tiles


def _box_diam(c):
    return float(np.sqrt(np.sum((c["hi"] - c["lo"]) ** 2)))


def _box_dist(a, b):
    g = np.maximum(0.0, np.maximum(a["lo"] - b["hi"], b["lo"] - a["hi"]))
    return float(np.sqrt(np.sum(g * g)))


CASES = [
    # (points, nu, ell, leaf, eta, aca_tol, k_cap)
    ("grid 24x20", 1.5, 0.2, 16, 1.0, 1e-8, 32),
    ("random 3D 1200", 0.5, 0.3, 24, 0.8, 1e-6, 24),
    ("grid 24x20 dense", 2.5, 0.2, 16, 0.0, 1e-8, 32),
]


def _points(name):
    if name.startswith("grid"):
        return synth.grid_points_2d(24, 20)
    return np.random.default_rng(synth.BASE_SEED + 77).uniform(size=(1200, 3))


@pytest.mark.parametrize("name,nu,ell,leaf,eta,tol,kcap", CASES)
def test_host_hmatrix_construction(dump_tool, tmp_path, name, nu, ell, leaf, eta, tol, kcap):
    pts = _points(name)
    n = pts.shape[0]
    sigma2 = 1.3
    perm, cl, far, near, tiles = _build(dump_tool, tmp_path, pts, nu, ell, sigma2, leaf, eta, tol, kcap)
    # cluster tree
    assert np.array_equal(np.sort(perm), np.arange(n))
    pc = pts[perm]
    assert cl[0]["b"] == 0 and cl[0]["e"] == n
    for c in cl:
        inside = pc[c["b"]:c["e"]]
        assert np.all(inside >= c["lo"] - 1e-15) and np.all(inside <= c["hi"] + 1e-15)
        c0, c1 = c["ch"]
        if c0 < 0:
            assert 0 < c["e"] - c["b"] <= leaf
        else:
            assert c["e"] - c["b"] > leaf
            assert cl[c0]["b"] == c["b"] and cl[c0]["e"] == cl[c1]["b"] and cl[c1]["e"] == c["e"]
    # exact kernel in cluster order (the oracle's Matern)
    G = covariance.dense_gamma(pc, nu, ell, sigma2)
    cover = np.zeros((n, n), dtype=np.int32)
    worst = 0.0
    for t, s, k, U, V in far:
        T, S = cl[t], cl[s]
        assert t != s and 1 <= k <= kcap
        assert min(_box_diam(T), _box_diam(S)) <= eta * _box_dist(T, S) * (1 + 1e-12)
        blk = G[T["b"]:T["e"], S["b"]:S["e"]]
        err = np.linalg.norm(blk - U @ V.T) / np.linalg.norm(blk)
        worst = max(worst, err)
        cover[T["b"]:T["e"], S["b"]:S["e"]] += 1
        cover[S["b"]:S["e"], T["b"]:T["e"]] += 1
    assert worst <= 10 * tol, worst
    for (t, s), tile in zip(near, tiles):
        T, S = cl[t], cl[s]
        assert T["ch"][0] < 0 and S["ch"][0] < 0 and t <= s
        np.testing.assert_allclose(tile, G[T["b"]:T["e"], S["b"]:S["e"]], rtol=1e-13, atol=0)
        cover[T["b"]:T["e"], S["b"]:S["e"]] += 1
        if t != s:
            cover[S["b"]:S["e"], T["b"]:T["e"]] += 1
    assert np.all(cover == 1)
    if eta == 0.0:
        assert not far
    else:
        assert far  # the compressed case really has low-rank blocks
    print(f"{name}: {len(far)} low-rank blocks (worst relative error {worst:.1e}), {len(near)} near tiles")
