"""torch.autograd.Function wrappers over the hand-written adjoints.

Each Function's forward and backward is one C-ABI call (see geraf.py); torch
only records the graph. Signals cross the wrappers as real views
[n_ant, n_f, 2] (re, im), so the incoming gradient is exactly
(dL/dRe s, dL/dIm s) — the g of the paper's adjoint formulas.
"""
import torch

from . import geraf as G


class FieldsMLP(torch.autograd.Function):
    """(params, xyz) -> (sdf [n], grad [3, n], refl [n]); gradient w.r.t. params."""

    @staticmethod
    def forward(ctx, params, xyz, field_kwargs):
        field = G.MLPField(params.detach(), **field_kwargs)
        sdf, grad, refl, saved = G.geraf_fields(field, xyz.detach(), keep_saved=True)
        ctx.field = field
        ctx.save_for_backward(xyz)
        ctx.saved_buf = saved
        return sdf, grad, refl

    @staticmethod
    def backward(ctx, d_sdf, d_grad, d_refl):
        (xyz,) = ctx.saved_tensors
        cont = lambda t: None if t is None else t.contiguous()
        d_params = G.geraf_fields_backward(ctx.field, xyz, ctx.saved_buf, cont(d_sdf), cont(d_grad), cont(d_refl))
        return d_params, None, None


class FieldsMLPOrigins(torch.autograd.Function):
    """SDF only at ray origins / antennas: stop-gradient by construction (section 6)."""

    @staticmethod
    def forward(ctx, params, xyz, field_kwargs):
        field = G.MLPField(params.detach(), **field_kwargs)
        sdf, _, _, _ = G.geraf_fields(field, xyz.detach(), want_grad=False, want_refl=False)
        return sdf

    @staticmethod
    def backward(ctx, d):
        return None, None, None


class Blend(torch.autograd.Function):
    """(sdf, refl, s, a_tx) -> (w, t_eff, c_ant, alpha, T); origin terms and
    alpha, T outputs carry no gradient (use w and t_eff downstream)."""

    @staticmethod
    def forward(ctx, sdf, refl, s, a_tx, sdf_apr, sdf_ant, n_ray, n_z):
        sv, av = float(s), float(a_tx)
        alpha, T, w, t_eff, c_ant = G.geraf_blend(sdf.detach(), refl.detach(), n_ray, n_z, sdf_apr.detach(),
                                                  sdf_ant.detach(), sv, av)
        ctx.save_for_backward(sdf, refl, alpha, T)
        ctx.meta = (n_ray, n_z, sv, av)
        ctx.mark_non_differentiable(c_ant, alpha, T)
        return w, t_eff, c_ant, alpha, T

    @staticmethod
    def backward(ctx, d_w, d_teff, _c, _a, _t):
        sdf, refl, alpha, T = ctx.saved_tensors
        n_ray, n_z, s, a_tx = ctx.meta
        cont = lambda t: None if t is None else t.contiguous()
        d_sdf, d_refl, d_sc = G.geraf_blend_backward(sdf, refl, alpha, T, n_ray, n_z, s, a_tx, cont(d_w),
                                                     cont(d_teff))
        need = ctx.needs_input_grad
        return (d_sdf, d_refl, d_sc[0] if need[2] else None, d_sc[1] if need[3] else None,
                None, None, None, None)


class Render(torch.autograd.Function):
    """(xyz, grad, w, t_eff, ant, c_ant) -> s as real view [n_ant, n_f, 2]."""

    @staticmethod
    def forward(ctx, xyz, grad, w, t_eff, ant, c_ant, band, directional):
        s = G.geraf_render(xyz.detach(), grad.detach(), w.detach(), t_eff.detach(), ant.detach(), c_ant.detach(),
                           band, directional)
        ctx.save_for_backward(xyz, grad, w, t_eff, ant, c_ant)
        ctx.band, ctx.directional = band, directional
        return torch.view_as_real(s)

    @staticmethod
    def backward(ctx, g):
        xyz, grad, w, t_eff, ant, c_ant = ctx.saved_tensors
        d_w, d_t, d_g = G.geraf_render_backward(xyz, grad, w, t_eff, ant, c_ant, ctx.band, g.contiguous(),
                                                ctx.directional)
        return None, d_g, d_w, d_t, None, None, None, None


class Filter(torch.autograd.Function):
    """s (real view [n_ant, n_f, 2]) -> heatmap P [n_vox]."""

    @staticmethod
    def forward(ctx, s, ant, vox, band):
        P, M, _, _ = G.geraf_filter(s.detach().contiguous(), ant, band, vox)
        ctx.save_for_backward(ant, vox, torch.view_as_real(M))
        ctx.band = band
        return P

    @staticmethod
    def backward(ctx, dP):
        ant, vox, M = ctx.saved_tensors
        g = G.geraf_filter_backward(ant, ctx.band, vox, M, dP.contiguous())
        return torch.view_as_real(g), None, None, None


def heatmap(params, xyz, apr, ant, vox, band, s, a_tx, n_ray, n_z, field_kwargs=None, directional=True):
    """Differentiable heatmap of an MLP field: fields -> blend -> render -> filter."""
    kw = field_kwargs or {}
    sdf, grad, refl = FieldsMLP.apply(params, xyz, kw)
    f_apr = FieldsMLPOrigins.apply(params, apr, kw)
    f_ant = FieldsMLPOrigins.apply(params, ant, kw)
    w, t_eff, c_ant, _, _ = Blend.apply(sdf, refl, s, a_tx, f_apr, f_ant, n_ray, n_z)
    sig = Render.apply(xyz, grad, w, t_eff, ant, c_ant, band, directional)
    return Filter.apply(sig, ant, vox, band)
