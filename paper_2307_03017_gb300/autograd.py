"""torch.autograd.Function over the hand-written warp + composite kernels.

Forward: ``reallife_render`` with the given cameras (Eq. eq_render with the over operator
of Eq. eq_over), ``[N][H][W][3]`` float32.  Backward: ``reallife_render_backward``, the
exact adjoint of warp and composite (dL/dc_d = T_d alpha_d g, dL/dalpha_d = T_d <c_d - B_d,
g>, bilinear transpose), with the per-plane transmittance recomputed from the MPI rather
than stored by the forward.  The MPI may be stored as float32 or bfloat16; the gradient is
accumulated in float32 and returned in the MPI's dtype.
"""
from __future__ import annotations

import torch

from . import Mpi, reallife_render, reallife_render_backward


class WarpComposite(torch.autograd.Function):
    @staticmethod
    def forward(ctx, M: torch.Tensor, near: float, far: float, ref, cams):
        m = Mpi(M.detach().contiguous(), near, far, ref)
        out = reallife_render(m, cams)
        ctx.save_for_backward(M)
        ctx.geometry = (near, far, ref, list(cams))
        return out

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        (M,) = ctx.saved_tensors
        near, far, ref, cams = ctx.geometry
        m = Mpi(M.detach().contiguous(), near, far, ref)
        g = reallife_render_backward(m, cams, grad_out.detach().float().contiguous())
        return g.to(M.dtype), None, None, None, None


def warp_composite(M: torch.Tensor, near: float, far: float, ref, cams) -> torch.Tensor:
    """Differentiable views ``[N][H][W][3]`` of the MPI ``M [D][H][W][4]`` for ``cams``."""
    return WarpComposite.apply(M, near, far, ref, cams)
