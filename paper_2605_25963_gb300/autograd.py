"""FEPE as a differentiable function of density scales (torch.autograd).

forward(scales) runs the transport with every solid of density group p scaled by
s_p and returns the full-energy-peak efficiency of each instance.  backward
replays the same histories (counter-based Philox streams make a replay exact)
in the score-accumulating kernel and returns
    dL/ds_p = sum_i dL/dFEPE_i * dFEPE_i/ds_p,
with dFEPE_i/ds_p the mean over histories of FEP * score_p, where
score_p = (collisions in group p)/s_p - sum over segments in group p of mu * length
(density-perturbation / differential-operator estimator).  No tracks are
stored; with ``fused=True`` the forward pass already runs the scoring kernel
and backward reuses its result.
"""
from __future__ import annotations

import numpy as np
import torch

from . import api


class FepeFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, scales, bvh, mats, items, opts_kw, fused):
        s = [float(v) for v in scales.detach().cpu().tolist()]
        n_group = len(s)
        inst = api.make_instances([(E, src, n, iid, s + list(sc[n_group:])) for E, src, n, iid, sc in items])
        opts = api.make_opts(n_group=n_group, **(opts_kw or {}))
        if fused:
            res, _, d, ds = api.gadep_grad(bvh, mats, inst, opts)
            ctx.dfepe = d
        else:
            res, _ = api.gadep_run_batch(bvh, mats, inst, opts)
            ctx.dfepe = None
        ctx.bvh, ctx.mats, ctx.inst, ctx.opts = bvh, mats, inst, opts
        ctx.scale_device, ctx.scale_dtype = scales.device, scales.dtype
        return torch.tensor([r["fepe"] for r in res], dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_out):
        d = ctx.dfepe
        if d is None:
            _, _, d, _ = api.gadep_grad(ctx.bvh, ctx.mats, ctx.inst, ctx.opts)
        g = grad_out.detach().cpu().numpy().astype(np.float64) @ d
        return (torch.as_tensor(g, dtype=ctx.scale_dtype, device=ctx.scale_device),
                None, None, None, None, None)


def fepe(scales, bvh, mats, items, opts_kw=None, fused=False):
    """items: [(energy, workloads.Source, n_hist, instance id, group scales)]."""
    return FepeFn.apply(scales, bvh, mats, items, opts_kw, fused)
