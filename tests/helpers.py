"""Shared test utilities: workloads from `synth`, and drivers that run the CUDA
path through the C-ABI binding (device buffers are torch CUDA tensors)."""

from __future__ import annotations

import numpy as np

import synth

# workload presets (sizes of the paper-shaped tomography workloads)
TINY = dict(grid=(32, 32), src=8, rec=4, steps=10, nu=1.5, ell=0.2, sigma2=1.0, noise=1e-4)
MEDIUM = dict(grid=(256, 256), src=20, rec=20, steps=50, nu=1.5, ell=0.1, sigma2=1.0, noise=1e-4)
LARGE = dict(grid=(512, 512), src=32, rec=32, steps=100, nu=0.5, ell=0.05, sigma2=1.0, noise=1e-4)


def workload(cfg, steps=None, seed_offset=0):
    steps = cfg["steps"] if steps is None else steps
    return synth.tomography_workload(cfg["grid"], cfg["src"], cfg["rec"], steps, cfg["ell"], cfg["sigma2"],
                                     cfg["noise"], seed=synth.BASE_SEED + seed_offset)


def lib():
    from paper_1405_2276_gb300 import fkf

    return fkf


def csr_tensors(h, device="cuda"):
    import torch

    return (torch.from_numpy(h.rowptr).to(device), torch.from_numpy(h.col).to(device),
            torch.from_numpy(h.val).to(device))


def run_filter(points, kernel, steps, precision=0, leaf=64, eta=1.0, aca_tol=1e-8, k_cap=32, trunc_tol=1e-12,
               m_max=None, r_max=None, want_W=False, want_var=True, ctx=None, hmat=None, refresh_every=0):
    """Run the GPU filter over steps = [(y, Csr, R (scalar or vector))].
    Returns (per-step dicts, context, hmatrix handle, filter handle)."""
    import torch

    fkf = lib()
    n = points.shape[0]
    own_ctx = ctx is None
    if own_ctx:
        ctx = fkf.fkf_create(0)
    if hmat is None:
        hmat = fkf.fkf_hmatrix_build(ctx, points, kernel[0], kernel[1], kernel[2], leaf=leaf, eta=eta,
                                     aca_tol=aca_tol, k_cap=k_cap, precision=precision)
    m_max = m_max or max(h.nrows for _, h, _ in steps)
    r_max = r_max or 2 * m_max
    f = fkf.fkf_filter_create(hmat, None, 0.0, trunc_tol, m_max, r_max)
    if refresh_every:
        fkf.fkf_filter_set_refresh(f, refresh_every)  # S10 scheduled by the library
    out = []
    dt = torch.float64 if precision == fkf.FKF_FP64 else torch.float32
    for k, (y, h, R) in enumerate(steps):
        Rv = None
        rs = 0.0
        if np.ndim(R) == 0:
            rs = float(R)
        else:
            Rv = np.ascontiguousarray(R, dtype=np.float64)
        nll = fkf.fkf_filter_step(f, np.ascontiguousarray(y, dtype=np.float64), h.nrows, h.rowptr, h.col, h.val,
                                  Rv, rs)
        st = fkf.fkf_filter_get(f, n)
        rec = dict(s=st["s"], alpha=st["alpha"], r=st["r"], D=st["D"].copy(), nll=nll)
        if want_var:
            v = torch.empty(n, dtype=torch.float64, device="cuda")
            fkf.fkf_variance(f, v)
            rec["var"] = v.cpu().numpy()
        if want_W and st["r"] > 0:
            W = torch.empty((n, st["r"]), dtype=dt, device="cuda")
            fkf.fkf_filter_get(f, n, want_s=False, want_D=False, W=W)
            rec["W"] = W.double().cpu().numpy()
        out.append(rec)
    return out, ctx, hmat, f


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
