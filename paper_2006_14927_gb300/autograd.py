"""torch.autograd binding of the telescope read-out and its adjoint kernel.

`telescope_readout(ctx, tracks, atm_params, seed, precision, sigma, nb)`
returns (D, Tbar): per telescope the Gaussian-smoothed photon density and
the mean arrival time of the bunches that land near its centre.  Gradients
flow to the 15 atmosphere parameters (a_0..a_4, b_0..b_4, c_0..c_4) and to
the step positions and directions (x0, y0, z0, ux, uy, uz); the backward
pass is the library's adjoint (cher_adjoint), which recomputes every
contributing bunch from its Philox counter instead of storing it.
"""
from __future__ import annotations

import torch

from ._binding import Context

_DIFF = ("x0", "y0", "z0", "ux", "uy", "uz")


def _atm_dict(params: torch.Tensor, template: dict) -> dict:
    v = params.detach().to("cpu", torch.float64).tolist()
    return dict(h_bound=list(template["h_bound"]), a=v[0:5], b=v[5:10], c=v[10:15],
                n0_minus_1=template["n0_minus_1"])


class _Readout(torch.autograd.Function):
    @staticmethod
    def forward(fctx, atm_params, x0, y0, z0, ux, uy, uz, ctx, fixed, seed, precision, sigma,
                nb, atm_template, state):
        atm = _atm_dict(atm_params, atm_template)
        if state.get("atm") != atm:                 # tables follow the parameters
            ctx.set_atmosphere(atm)
            state["atm"] = atm
        dev = dict(fixed)
        dev.update(x0=x0.detach().contiguous(), y0=y0.detach().contiguous(),
                   z0=z0.detach().contiguous(), ux=ux.detach().contiguous(),
                   uy=uy.detach().contiguous(), uz=uz.detach().contiguous())
        D, T = ctx.density(dev, seed, precision, sigma, nb)
        fctx.ctx, fctx.dev, fctx.seed, fctx.precision = ctx, dev, seed, precision
        fctx.sigma, fctx.nb = sigma, nb
        fctx.dtypes = (atm_params.dtype, x0.dtype, ux.dtype)
        fctx.devices = (atm_params.device, x0.device, ux.device)
        return D, T

    @staticmethod
    def backward(fctx, gD, gT):
        ctx = fctx.ctx
        ga, gt = ctx.adjoint(fctx.dev, fctx.seed, fctx.precision,
                             gD.detach().to(torch.float64), gT.detach().to(torch.float64),
                             fctx.sigma, fctx.nb)
        da, dp, dd = fctx.dtypes
        va, vp, vd = fctx.devices
        grads = [gt[m].to(device=vp if m < 3 else vd, dtype=dp if m < 3 else dd)
                 for m in range(6)]
        return (ga.to(device=va, dtype=da), *grads, None, None, None, None, None, None, None,
                None)


def telescope_readout(ctx: Context, tracks: dict, atm_params: torch.Tensor, atm_template: dict,
                      seed: int, precision: int, sigma: float = 1.0, nb=None, state=None):
    """(D, Tbar) with autograd.  `tracks` holds device tensors of the ABI's
    dtypes; the six differentiable fields are taken from it (they may require
    grad).  `state` (a dict kept by the caller) remembers the atmosphere the
    context's tables were built for."""
    state = {} if state is None else state
    fixed = {k: v for k, v in tracks.items() if k not in _DIFF}
    return _Readout.apply(atm_params, *(tracks[k] for k in _DIFF), ctx, fixed, seed, precision,
                          sigma, nb, atm_template, state)
