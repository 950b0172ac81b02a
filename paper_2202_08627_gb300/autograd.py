"""PyTorch autograd wrappers over the C ABI.

EIObjective: S (Eq. 5) of every slice as a differentiable function of the
physical volume; one ei_objective_grad call computes S and its analytic
gradient together, the gradient is kept for backward.

EIProject: the Radon transform R (Eq. 1) of the three channels, whose backward
is the library's gather-form transpose R^T (ei_backproject), so losses can
flow through the projector.

Layouts are the library's (see include/ei.h): a volume is a [vol_count, 4]
float32 CUDA tensor (mu, delta, sigma, pad per voxel), projections a flat
[proj_count] tensor of 3 planes per slice.  The chain rule's scaling by the
upstream gradient and the planar-to-interleaved reordering of projection
gradients are plain tensor operations; the projector, the IC model, the
residual, the gradient and the adjoint all run in libei.so.
"""
from __future__ import annotations

import torch

from . import ei


def _slice_index(geom: ei.Geometry, device) -> torch.Tensor:
    """Slice number of every voxel in the vol layout (cached on the geometry)."""
    key = "_voxel_slice_" + str(device)
    idx = getattr(geom, key, None)
    if idx is None:
        counts = torch.tensor([sl.vol_count for sl in geom.slices], device=device)
        idx = torch.repeat_interleave(torch.arange(geom.n_slices, device=device), counts)
        setattr(geom, key, idx)
    return idx


class EIObjective(torch.autograd.Function):
    """S = EIObjective.apply(vol, geom, s_exp) -> float64 tensor [n_slices]."""

    @staticmethod
    def forward(ctx, vol, geom, s_exp):
        vol = vol.contiguous()
        S = torch.zeros(geom.n_slices, dtype=torch.float64, device=vol.device)
        grad = torch.empty_like(vol) if vol.requires_grad else None
        ei.ei_objective_grad(geom, vol, s_exp, S, grad)
        ctx.geom = geom
        ctx.save_for_backward(grad if grad is not None else torch.empty(0, device=vol.device))
        return S

    @staticmethod
    def backward(ctx, gS):
        (grad,) = ctx.saved_tensors
        if grad.numel() == 0:
            return None, None, None
        geom = ctx.geom
        if geom.n_slices == 1:
            scale = gS.to(grad.dtype).reshape(1, 1)
        else:
            scale = gS.to(grad.dtype)[_slice_index(geom, grad.device)].unsqueeze(1)
        return grad * scale, None, None


def _proj_to_sino4(geom: ei.Geometry, g: torch.Tensor) -> torch.Tensor:
    """Projection-layout tensor (3 planes per slice) -> sino4 layout."""
    out = torch.zeros((geom.sino4_count, 4), dtype=torch.float32, device=g.device)
    for sl in geom.slices:
        planes = g[sl.proj_offset:sl.proj_offset + sl.proj_count].view(3, sl.n_theta * sl.n_dp)
        out[sl.sino4_offset:sl.sino4_offset + sl.sino4_count, :3] = planes.t()
    return out


class EIProject(torch.autograd.Function):
    """proj = EIProject.apply(vol, geom): R of the three channels."""

    @staticmethod
    def forward(ctx, vol, geom):
        vol = vol.contiguous()
        proj = torch.empty(geom.proj_count, dtype=torch.float32, device=vol.device)
        ei.ei_project(geom, vol, proj)
        ctx.geom = geom
        return proj

    @staticmethod
    def backward(ctx, gproj):
        geom = ctx.geom
        out = torch.empty((geom.vol_count, 4), dtype=torch.float32, device=gproj.device)
        ei.ei_backproject(geom, _proj_to_sino4(geom, gproj.contiguous()), out)
        return out, None


def objective(vol, geom, s_exp):
    return EIObjective.apply(vol, geom, s_exp)


def project(vol, geom):
    return EIProject.apply(vol, geom)
