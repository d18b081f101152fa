"""torch.autograd wrappers over the C-ABI (hand-written adjoints).

HApply     Y = Gamma_H X (original point order).  Backward:
           fkf_hmatrix_apply_adjoint, i.e. the adjoint apply Gamma_H^T dY (the
           same sweep: Gamma_H is exactly symmetric) and d/dsigma2 =
           <dY, Y> / sigma2 (Gamma_H = sigma2 * Gamma_1,H), both in the library.
FilterNLL  summed innovation NLL of K filter steps with a fixed H and its
           gradient with respect to the measurements, the prior mean, the
           Matern variance and the noise variance, from fkf_nll_gradient
           (reverse-mode data-space recursion in the library).

All products and reductions run in libfkf.so; this module only moves tensors
across the C-ABI and scales the library's gradients by the incoming scalar
gradient of FilterNLL.
"""

from __future__ import annotations

import numpy as np
import torch

from . import fkf


class HApply(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, sigma2, hmat):
        Xc = X.contiguous()
        Y = torch.empty_like(Xc)
        fkf.fkf_hmatrix_apply(hmat, Xc, Y)
        ctx.save_for_backward(Y)
        ctx.hmat = hmat
        ctx.sigma2 = float(sigma2)
        return Y

    @staticmethod
    def backward(ctx, gY):
        (Y,) = ctx.saved_tensors
        gYc = gY.contiguous()
        gX = torch.empty_like(gYc)
        g_sigma2 = fkf.fkf_hmatrix_apply_adjoint(ctx.hmat, gYc, Y, gX)
        return gX, torch.tensor(g_sigma2, dtype=torch.float64), None


class FilterNLL(torch.autograd.Function):
    """nll = FilterNLL.apply(y, s0, sigma2, rho, hmat, H, alpha0)
    y: (K, m) float64; s0: (N,) float64; sigma2, rho: 0-d float64 tensors
    (sigma2 must be the variance the H-matrix was built with); H: a CSR
    operator with rowptr/col/val numpy arrays."""

    @staticmethod
    def forward(ctx, y, s0, sigma2, rho, hmat, H, alpha0=0.0):
        y_np = np.ascontiguousarray(y.detach().cpu().numpy(), dtype=np.float64)
        s0_np = np.ascontiguousarray(s0.detach().cpu().numpy(), dtype=np.float64)
        nll, gy, gs0, gsig, grho = fkf.fkf_nll_gradient(hmat, y_np, H.rowptr, H.col, H.val, float(rho), s0_np,
                                                        float(alpha0))
        ctx.grads = (torch.from_numpy(gy).to(y.device), torch.from_numpy(gs0).to(s0.device),
                     torch.tensor(gsig, dtype=torch.float64), torch.tensor(grho, dtype=torch.float64))
        return torch.tensor(nll, dtype=torch.float64)

    @staticmethod
    def backward(ctx, g):
        gy, gs0, gsig, grho = ctx.grads
        g = g.detach().cpu().to(torch.float64)
        return g.to(gy.device) * gy, g.to(gs0.device) * gs0, g * gsig, g * grho, None, None, None
