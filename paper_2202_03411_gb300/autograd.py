"""torch.autograd.Function over scatman_forward / scatman_backward.

The differentiable parameters of a shape are packed into one float64 vector in
the order the C ABI's gradient uses:
  sphere     [r, delta, beta]
  ellipsoid  [a, b, c, delta, beta]
  harmonics  [a_lm for l >= 1 (index l*l+l+m - 1), R0, delta, beta]
Orientation and centre are held fixed.  The forward pass runs the library's
voxeliser and contraction; the backward pass runs its adjoint kernels, which
recompute occupancy and transmission from the shape.  A handle caches the
field of its last forward call, so give each in-flight fit its own handle.
"""
from __future__ import annotations

import copy

import numpy as np
import torch

from . import api
from .types import ELLIPSOID, SPHERE, Shape, alm_array


def params_of(shape: Shape) -> np.ndarray:
    if shape.kind == SPHERE:
        v = [shape.r]
    elif shape.kind == ELLIPSOID:
        v = [shape.a, shape.b, shape.c]
    else:
        v = list(alm_array(shape)[1:]) + [shape.R0]
    return np.array(v + [shape.delta, shape.beta], dtype=np.float64)


def shape_with(template: Shape, params) -> Shape:
    p = np.asarray(params, dtype=np.float64)
    s = copy.deepcopy(template)
    if s.kind == SPHERE:
        s.r = float(p[0])
    elif s.kind == ELLIPSOID:
        s.a, s.b, s.c = (float(x) for x in p[:3])
    else:
        n = (s.lmax + 1) ** 2 - 1
        alm = np.zeros(n + 1)
        alm[1:] = p[:n]
        s.alm = alm
        s.R0 = float(p[n])
    s.delta, s.beta = float(p[-2]), float(p[-1])
    return s


class MSFTFunction(torch.autograd.Function):
    """I = |A(params)|^2 on the handle's detector; grad flows to params."""

    @staticmethod
    def forward(ctx, params: torch.Tensor, handle: api.Handle, template: Shape):
        shape = shape_with(template, params.detach().cpu().numpy())
        api.scatman_voxelise(handle, shape)
        n = api.scatman_n_pix(handle)
        dt = torch.float64 if handle.fp64 else torch.float32
        I = torch.empty(n, dtype=dt, device="cuda")
        api.scatman_forward(handle, I)
        ctx.handle = handle
        ctx.pdevice = params.device
        return I

    @staticmethod
    def backward(ctx, grad_I: torch.Tensor):
        dt = torch.float64 if ctx.handle.fp64 else torch.float32
        g = api.scatman_backward(ctx.handle, grad_I.detach().to(device="cuda", dtype=dt).contiguous())
        return torch.from_numpy(g).to(ctx.pdevice), None, None


def msft(params: torch.Tensor, handle: api.Handle, template: Shape) -> torch.Tensor:
    return MSFTFunction.apply(params, handle, template)
