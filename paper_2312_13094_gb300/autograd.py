"""torch.autograd binding of forward modelling: receivers as a function of the
squared slowness m = 1/v^2 (Eq. 1, App. A), with the checkpointed adjoint of
libfd.so as the backward pass.

Both passes run in libfd.so: the forward pass is fd_set_model(m) + fd_forward,
the backward pass is fd_backward (the transpose of d rec / d m applied to the
incoming receiver gradient, recomputing the forward states from checkpoints).
This module only moves tensors between autograd and those two calls.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as fd


class AcousticModelling(torch.autograd.Function):
    """rec = F(m) for one shot on `grid` (a binding.Grid).

    m: physical squared slowness, float32 [nz][ny][nx] in (ms/m)^2 (1/v^2 with v
    in km/s), on the grid's device.  src / rec: point coordinates in metres
    ([n][3], x y z).  wavelet: [nt][n_src] float32.  Returns [nt][n_rec].
    The grid's model is replaced by m in both passes.
    """

    @staticmethod
    def forward(ctx, m, grid, src, wavelet, rec, n_checkpoints):
        m = m.detach().contiguous()
        if m.dtype != torch.float32:
            raise TypeError("m must be float32")
        if tuple(m.shape) != grid.phys_shape:
            raise ValueError(f"m has shape {tuple(m.shape)}, grid needs {grid.phys_shape}")
        grid.set_model(m, fd.FD_MODEL_M)
        out = torch.zeros((grid.nt, len(rec)), device=m.device, dtype=torch.float32)
        wav = torch.as_tensor(np.ascontiguousarray(wavelet, np.float32)).to(m.device)
        fd.check(grid.forward(src, wav, rec, out), "fd_forward")
        ctx.save_for_backward(m)
        ctx.grid, ctx.src, ctx.wav, ctx.rec = grid, src, wav, rec
        ctx.n_checkpoints = int(n_checkpoints)
        return out

    @staticmethod
    def backward(ctx, grad_rec):
        (m,) = ctx.saved_tensors
        grid = ctx.grid
        grid.set_model(m, fd.FD_MODEL_M)
        grad_m = torch.zeros_like(m)
        fd.check(grid.backward(ctx.src, ctx.wav, ctx.rec, grad_rec.detach().contiguous(),
                               ctx.n_checkpoints, grad_m), "fd_backward")
        return grad_m, None, None, None, None, None


def modelling(m, grid, src, wavelet, rec, n_checkpoints=10):
    """Differentiable receivers of one shot (see AcousticModelling)."""
    return AcousticModelling.apply(m, grid, src, wavelet, rec, n_checkpoints)
