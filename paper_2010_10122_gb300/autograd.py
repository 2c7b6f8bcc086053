"""torch.autograd Functions over the w-gridding operator.

R maps a real image to complex visibilities and is R-linear (Sec. 2: "R is an R-linear map");
its adjoint with respect to the real inner product on images and Re<.,.> on visibilities
(Sec. 5.1, Eq. adjointness) is R^dagger = grid.  PyTorch hands a complex output's backward
the gradient dL/dRe(y) + i dL/dIm(y); for y = R x with real x the chain rule gives
dL/dx = Re(R^H g) = R^dagger(g), so the backward of degrid is one grid call, and the backward of
grid is one degrid call.  Neither Function keeps activations: only the plan (resident) and the
optional weights are referenced by the graph.
"""
from __future__ import annotations

import torch


class WDegrid(torch.autograd.Function):
    """vis = R(x) (wg_degrid) with dL/dx = R^dagger(dL/dvis) (wg_grid)."""

    @staticmethod
    def forward(ctx, x, plan, wgt=None):
        ctx.plan = plan
        ctx.wgt = wgt
        return plan.degrid(x.contiguous(), wgt=wgt)

    @staticmethod
    def backward(ctx, g):
        gx = ctx.plan.grid(g.contiguous(), wgt=ctx.wgt) if ctx.needs_input_grad[0] else None
        return gx, None, None


class WGrid(torch.autograd.Function):
    """image = R^dagger(vis) (wg_grid) with dL/dvis = R(dL/dimage) (wg_degrid)."""

    @staticmethod
    def forward(ctx, vis, plan, wgt=None):
        ctx.plan = plan
        ctx.wgt = wgt
        return plan.grid(vis.contiguous(), wgt=wgt)

    @staticmethod
    def backward(ctx, g):
        gv = ctx.plan.degrid(g.contiguous(), wgt=ctx.wgt) if ctx.needs_input_grad[0] else None
        return gv, None, None


def degrid(x, plan, wgt=None):
    return WDegrid.apply(x, plan, wgt)


def grid(vis, plan, wgt=None):
    return WGrid.apply(vis, plan, wgt)
