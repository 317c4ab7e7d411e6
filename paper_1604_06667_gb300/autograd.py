"""Differentiable gridding: ``torch.autograd.Function`` over the C ABI.

    R = grid(gridder, lon, lat, data, sigma)      # Eq. 3 map [P, C]
    loss(R).backward()                           # dL/ddata = G^T dL/dR (cg_degrid),
                                                 # dL/dsigma (cg_grid_dsigma)

The forward pass is ``cg_grid_oneshot``; the backward pass runs the adjoint
(degridding) of the same normalised operator R = G D, G[p][n] =
omega_n w_pn / W_p, and the width derivative for the circular kernel with the
support held fixed.  All arithmetic runs in the CUDA library.
"""
from __future__ import annotations

import torch


class GridFunction(torch.autograd.Function):
    """R = G(sigma) D.  Inputs: data [N, C] float32 (differentiable), sigma
    0-d tensor in degrees (differentiable; gauss1d), plus the non-tensor
    gridder, coordinates, support and hpx_maxres."""

    @staticmethod
    def forward(ctx, data, sigma, gridder, lon, lat, support, hpx_maxres):
        s = float(sigma)
        if getattr(gridder, "_sigma", None) != (s, support, hpx_maxres):
            gridder.set_kernel("gauss1d", (s,), support, hpx_maxres)
            gridder._sigma = (s, support, hpx_maxres)
        W = torch.empty(gridder.n_targets, device=gridder.device, dtype=torch.float32)
        R = gridder.grid_oneshot(lon, lat, data.detach().float().contiguous(), out_weights=W)
        ctx.gridder = gridder
        ctx.gen = gridder.index_gen
        ctx.save_for_backward(data, W)
        return R

    @staticmethod
    def backward(ctx, grad_R):
        data, W = ctx.saved_tensors
        g = ctx.gridder
        if g.index_gen != ctx.gen:
            raise RuntimeError("the gridder indexed other samples since this forward pass; "
                               "run backward first")
        grad_R = torch.nan_to_num(grad_R.float(), nan=0.0).contiguous()
        grad_data = grad_sigma = None
        if ctx.needs_input_grad[0]:
            grad_data = g.degrid(grad_R, map_weights=W).to(data.dtype)
        if ctx.needs_input_grad[1]:
            _, ds = g.dsigma(data.detach().float(), grad_out=grad_R, want_dR=False)
            grad_sigma = ds.to(torch.float32)
        return grad_data, grad_sigma, None, None, None, None, None


def grid(gridder, lon, lat, data, sigma, support, hpx_maxres=None):
    """Differentiable one-shot gridding with a circular Gaussian of width
    ``sigma`` (degrees, tensor) and fixed support (degrees)."""
    if not isinstance(sigma, torch.Tensor):
        sigma = torch.tensor(float(sigma), device=gridder.device)
    return GridFunction.apply(data, sigma, gridder, lon, lat, float(support),
                              float(hpx_maxres or float(sigma) / 2.0))
