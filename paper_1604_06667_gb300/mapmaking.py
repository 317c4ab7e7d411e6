"""Map making by gradient descent on the adjoint of the gridding operator.

Find the map m [P, C] whose interpolation to the sample positions reproduces
the samples: minimise L(m) = 1/2 ||G^T m - D||^2, with G the normalised
gridding operator of Eq. 3 (R = G D) and G^T its adjoint (cg_degrid).  The
gradient is G (G^T m - D): one degridding and one gridding per step (the
gridding reuses the sample index of the first call).  Step 1/max_n sum_p
G[p][n] (G^T applied to a map of ones): with the unit row sums of Eq. 3 this
bounds ||G G^T||_2, so the loss never increases.
"""
from __future__ import annotations

import torch

from . import _capi as C


def gd(gridder, lon, lat, data, steps: int = 50, alpha: float | None = None):
    """Returns (m [P, C], losses [steps + 1] float64 on the host, alpha)."""
    P, Cc = gridder.n_targets, gridder.n_channels
    dev = gridder.device
    D = torch.as_tensor(data, device=dev, dtype=torch.float32).reshape(-1, Cc).contiguous()
    W = torch.empty(P, device=dev, dtype=torch.float32)
    g = torch.empty((P, Cc), device=dev, dtype=torch.float32)
    gridder.grid_oneshot(lon, lat, D, out=g, out_weights=W)      # sample index + W_p
    if alpha is None:
        colsum = gridder.degrid(torch.ones((P, Cc), device=dev), map_weights=W)[:, 0]
        alpha = 1.0 / float(colsum.max())
    m = torch.zeros((P, Cc), device=dev, dtype=torch.float32)
    losses = torch.empty(steps + 1, device=dev, dtype=torch.float64)
    h = gridder._h
    for k in range(steps + 1):
        r = gridder.degrid(m, map_weights=W)                     # G^T m
        # r <- G^T m - D and the loss 1/2 |r|^2 (FP64), in the library
        C.cg_md_residual(h, r.data_ptr(), D.data_ptr(), r.numel(), losses[k:].data_ptr())
        if k == steps:
            break
        gridder.grid_oneshot(None, None, r, out=g)               # G r, same samples
        C.cg_md_update(h, m.data_ptr(), g.data_ptr(), float(alpha), m.numel())
    return m, losses.cpu().numpy(), alpha
