"""torch.autograd.Function over the GPU adjoint: the sum of per-SNP Wald
chi2 statistics as a differentiable function of the heritability h and the
phenotype y.  Forward and backward both run in the library's kernels
(gwas_adjoint_block); this module only moves arguments."""
from __future__ import annotations

import numpy as np
import torch

from . import GLS


class WaldChi2Sum(torch.autograd.Function):
    """loss = sum_i chi2_i(h, y) over the SNP blocks; d loss/dh and d loss/dy
    come from one adjoint pass per block (computed during forward).

    Every forward call sets the study up afresh for its (h, y): M and its
    Cholesky factor depend on h, and y~, r_T and the solve constants on y, so
    a call pays gwas_init (the FP64 Cholesky, n^3/3 flop, plus in the split
    precisions the formation of L^-1 on the tensor cores) before its blocks:
    about 0.1-0.5 s at n = 5,000-10,000, against milliseconds per block.  A fit
    that moves h re-factors M at every step anyway; callers that evaluate many
    blocks at one (h, y) should pass them all in one call."""

    @staticmethod
    def forward(ctx, h, y, phi, XL, blocks, sigma2=1.0, bs=4096, precision="fp64"):
        hv = float(h.detach().cpu())
        yv = y.detach().to("cpu", torch.float64).numpy()
        dh = np.zeros(1)
        dy = np.zeros(yv.shape[0])
        total = 0.0
        with GLS(phi, XL, yv, hv, sigma2, bs=bs, precision=precision) as g:
            for X in blocks:
                chi2, _, dh, dy = g.adjoint_block(X, dh_accum=dh, dy_accum=dy)
                total += float(np.nansum(chi2))
        ctx.save_for_backward(torch.tensor(dh[0], dtype=torch.float64), torch.from_numpy(dy))
        ctx.y_device = y.device
        return torch.tensor(total, dtype=torch.float64, device=h.device)

    @staticmethod
    def backward(ctx, grad_out):
        dh, dy = ctx.saved_tensors
        g = grad_out.detach().to("cpu", torch.float64)
        return (g * dh).to(grad_out.device), (g * dy).to(ctx.y_device), None, None, None, None, None, None


def wald_chi2_sum(h, y, phi, XL, blocks, sigma2: float = 1.0, bs: int = 4096, precision: str = "fp64"):
    """precision: "fp64", or "bf16x3" / "tf32x3" (the block solve and the
    transpose solve on the tensor cores; the per-SNP adjoint arithmetic FP64)."""
    return WaldChi2Sum.apply(h, y, phi, XL, blocks, sigma2, bs, precision)
