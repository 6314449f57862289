"""torch.autograd.Function around flood_adjoint: the gauge-misfit loss of an
ensemble as a differentiable function of the base Manning field, the
members' rain multipliers and their initial depths (the paper has no
adjoint; this serves gradient calibration beside the particle filter).

Forward and reverse sweeps both run in the library's CUDA kernels; this
module only moves tensors across the C ABI."""
from __future__ import annotations

import numpy as np
import torch

from . import capi


class GaugeMisfit(torch.autograd.Function):
    """loss = sum_i sum_s sum_k (h_i(t_s)[cell_k] - d[s][k])^2 over members i,
    observation times t_s = s * sample_dt and gauges k."""

    @staticmethod
    def forward(ctx, n_base, rain_mult, h0, z, scale, hyetograph, cells, d, sample_dt,
                params=None, ckpt_every=0):
        M = int(rain_mult.shape[0])
        ny, nx = int(z.shape[0]), int(z.shape[1])
        zz = z.detach().to(torch.float32).contiguous()
        nn = n_base.detach().to(torch.float32).contiguous()
        with capi.Grid(zz, nn, params) as g:
            h0c = h0.detach().to(torch.float32).contiguous()
            if h0c.dim() == 2:
                h0c = h0c.expand(M, ny, nx).contiguous()
            g.ensemble_init(M, rain_mult.detach().to(torch.float32).contiguous(),
                            scale.detach().to(torch.float32).contiguous(),
                            hyetograph.detach().to(torch.float32).contiguous(), h0=h0c)
            out = g.adjoint(np.asarray(cells, np.int32), np.asarray(d, np.float64), sample_dt,
                            ckpt_every=ckpt_every)
        dev = n_base.device
        ctx.save_for_backward(torch.from_numpy(out["grad_n"]).to(dev),
                              torch.from_numpy(out["grad_rain"]).to(dev, torch.float64),
                              torch.from_numpy(out["grad_h0"]).to(dev))
        ctx.h0_dim = h0.dim()
        ctx.dtypes = (n_base.dtype, rain_mult.dtype, h0.dtype)
        return torch.tensor(float(out["loss"].sum()), dtype=torch.float64, device=dev)

    @staticmethod
    def backward(ctx, gout):
        gn, gr, gh = ctx.saved_tensors
        g = gout.to(torch.float64)
        dn = (g * gn.to(torch.float64)).to(ctx.dtypes[0])
        drm = (g * gr).to(ctx.dtypes[1])
        dh = g * gh.to(torch.float64)
        if ctx.h0_dim == 2:
            dh = dh.sum(dim=0)
        return dn, drm, dh.to(ctx.dtypes[2]), None, None, None, None, None, None, None, None


def gauge_misfit(n_base, rain_mult, h0, z, scale, hyetograph, cells, d, sample_dt, params=None,
                 ckpt_every=0):
    return GaugeMisfit.apply(n_base, rain_mult, h0, z, scale, hyetograph, cells, d, sample_dt,
                             params, ckpt_every)


class LandGaugeMisfit(torch.autograd.Function):
    """The same loss with land cover (Section 4.1): differentiable in every
    member's Manning n of each class, its drainage rate, its rain multiplier
    and its initial depth (flood_adjoint with flood_adjoint_land_grad)."""

    @staticmethod
    def forward(ctx, n_class, drain_rate, rain_mult, h0, z, n_base, cls, classes, scale,
                hyetograph, cells, d, sample_dt, params=None, ckpt_every=0):
        M = int(rain_mult.shape[0])
        ny, nx = int(z.shape[0]), int(z.shape[1])
        zz = z.detach().to(torch.float32).contiguous()
        nn = n_base.detach().to(torch.float32).contiguous()
        with capi.Grid(zz, nn, params) as g:
            g.set_land_cover(np.asarray(cls, np.uint8), classes)
            h0c = h0.detach().to(torch.float32).contiguous()
            if h0c.dim() == 2:
                h0c = h0c.expand(M, ny, nx).contiguous()
            g.ensemble_init(M, rain_mult.detach().to(torch.float32).contiguous(),
                            scale.detach().to(torch.float32).contiguous(),
                            hyetograph.detach().to(torch.float32).contiguous(), h0=h0c)
            g.set_land_params(n_class.detach().to("cpu", torch.float32).numpy(),
                              drain_rate.detach().to("cpu", torch.float32).numpy())
            out = g.adjoint(np.asarray(cells, np.int32), np.asarray(d, np.float64), sample_dt,
                            ckpt_every=ckpt_every)
            gc, gd = g.adjoint_land_grad()
        dev = rain_mult.device
        ctx.save_for_backward(torch.from_numpy(gc).to(dev), torch.from_numpy(gd).to(dev),
                              torch.from_numpy(out["grad_rain"]).to(dev, torch.float64),
                              torch.from_numpy(out["grad_h0"]).to(dev))
        ctx.h0_dim = h0.dim()
        ctx.dtypes = (n_class.dtype, drain_rate.dtype, rain_mult.dtype, h0.dtype)
        return torch.tensor(float(out["loss"].sum()), dtype=torch.float64, device=dev)

    @staticmethod
    def backward(ctx, gout):
        gc, gd, gr, gh = ctx.saved_tensors
        g = gout.to(torch.float64)
        dh = g * gh.to(torch.float64)
        if ctx.h0_dim == 2:
            dh = dh.sum(dim=0)
        return ((g * gc).to(ctx.dtypes[0]), (g * gd).to(ctx.dtypes[1]),
                (g * gr).to(ctx.dtypes[2]), dh.to(ctx.dtypes[3])) + (None,) * 11


def land_gauge_misfit(n_class, drain_rate, rain_mult, h0, z, n_base, cls, classes, scale,
                      hyetograph, cells, d, sample_dt, params=None, ckpt_every=0):
    return LandGaugeMisfit.apply(n_class, drain_rate, rain_mult, h0, z, n_base, cls, classes,
                                 scale, hyetograph, cells, d, sample_dt, params, ckpt_every)
