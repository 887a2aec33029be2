"""One pass of the rendering hot path, forward and adjoint, through the C ABI.

sample -> fields (+ ray-origin and antenna SDF) -> lensless blend -> render ->
matched filter + L2 heatmap loss -> filter adjoint -> render adjoint ->
blend adjoint -> fields adjoint (MLP parameter gradient). Every step is a call
into libgeraf.so on the current CUDA stream; this module only wires tensors.
"""
from dataclasses import dataclass
from typing import Optional

import numpy as np
import torch

from . import geraf as G

# kernel launches made by one call of each entry point (for launch accounting)
LAUNCHES = {"sample": 1, "fields": 1, "blend": 2, "render": 4, "filter": 4, "filter_backward": 4,
            "render_backward": 4, "blend_backward": 2}


def fields_backward_launches(n_hidden: int) -> int:
    return n_hidden + 2


@dataclass
class Geometry:
    grid: object                 # GerafGrid of the sample points
    n_ray: int
    n_z: int
    ant: torch.Tensor            # [3, n_ant]
    vox: torch.Tensor            # [3, n_vox] heatmap voxel centres
    band: G.Band
    sharpness: float
    a_tx: float
    mode: int


def make_geometry(wl, device="cuda") -> Geometry:
    """Device-side geometry of a workload description (geraf_inputs.Workload)."""
    from geraf_inputs import antenna_array
    g = wl.grid
    grid = G.make_grid(g.lo, g.pitch, g.n, g.aperture_z)
    h = wl.heat
    hgrid = G.make_grid(h.lo, h.pitch, h.n, h.aperture_z)
    vox, _ = G.geraf_sample(hgrid, G.SAMPLE_UNIFORM, device=device)
    ant = torch.as_tensor(antenna_array(wl.array_n, wl.array_n, wl.array_pitch), device=device)
    f_hi = 81e9
    band = G.Band(77e9, (f_hi - 77e9) / (wl.n_f - 1), wl.n_f)
    return Geometry(grid, g.n_ray, g.n[2], ant, vox, band, float(wl.sharpness), float(wl.a_tx), wl.sample_mode)


def render_heatmap(geo: Geometry, field, mode=G.SAMPLE_UNIFORM, seed=0, step=0, extra=None):
    """Forward only: heatmap P of a field (used to make synthetic targets).
    `extra` = (xyz [3, m], w [m]) isotropic point reflectors appended with T' = 1."""
    xyz, apr = G.geraf_sample(geo.grid, mode, seed, step, device=geo.ant.device)
    f, grad, a, _ = G.geraf_fields(field, xyz)
    fa, _, _, _ = G.geraf_fields(field, apr, want_grad=False, want_refl=False)
    fn, _, _, _ = G.geraf_fields(field, geo.ant, want_grad=False, want_refl=False)
    alpha, T, w, t_eff, c_ant = G.geraf_blend(f, a, geo.n_ray, geo.n_z, fa, fn, geo.sharpness, geo.a_tx)
    if extra is not None:
        ex, ew = extra
        m = ex.shape[1]
        xyz = torch.cat([xyz, ex], 1).contiguous()
        grad = torch.cat([grad, torch.zeros(3, m, device=xyz.device)], 1).contiguous()
        w = torch.cat([w, ew]).contiguous()
        t_eff = torch.cat([t_eff, torch.full((m,), 2.0, device=xyz.device)]).contiguous()
    s = G.geraf_render(xyz, grad, w, t_eff, geo.ant, c_ant, geo.band)
    P, M, _, _ = G.geraf_filter(s, geo.ant, geo.band, geo.vox)
    return P, s


@dataclass
class StepResult:
    loss: torch.Tensor           # 0-d float64 (device)
    d_params: Optional[torch.Tensor]
    d_scalars: torch.Tensor      # (dL/ds, dL/dA'_tx)
    P: torch.Tensor


def forward_backward(geo: Geometry, field, target: torch.Tensor, seed: int, step: int, timers=None) -> StepResult:
    """One hot-path pass (all forward steps and their adjoints). `timers` may map
    a step name to a pair of CUDA events recorded around that call."""
    def tic(name):
        if timers is not None and name in timers:
            timers[name][0].record()

    def toc(name):
        if timers is not None and name in timers:
            timers[name][1].record()

    xyz, apr = G.geraf_sample(geo.grid, geo.mode, seed, step, device=geo.ant.device)
    is_mlp = isinstance(field, G.MLPField)
    f, grad, a, saved = G.geraf_fields(field, xyz, keep_saved=is_mlp)
    fa, _, _, _ = G.geraf_fields(field, apr, want_grad=False, want_refl=False)
    fn, _, _, _ = G.geraf_fields(field, geo.ant, want_grad=False, want_refl=False)
    alpha, T, w, t_eff, c_ant = G.geraf_blend(f, a, geo.n_ray, geo.n_z, fa, fn, geo.sharpness, geo.a_tx)
    tic("render")
    s = G.geraf_render(xyz, grad, w, t_eff, geo.ant, c_ant, geo.band)
    toc("render")
    tic("filter")
    P, M, loss, dP = G.geraf_filter(s, geo.ant, geo.band, geo.vox, target)
    toc("filter")
    tic("filter_backward")
    g_s = G.geraf_filter_backward(geo.ant, geo.band, geo.vox, M, dP)
    toc("filter_backward")
    tic("render_backward")
    d_w, d_t, d_G = G.geraf_render_backward(xyz, grad, w, t_eff, geo.ant, c_ant, geo.band, g_s)
    toc("render_backward")
    d_f, d_a, d_sc = G.geraf_blend_backward(f, a, alpha, T, geo.n_ray, geo.n_z, geo.sharpness, geo.a_tx, d_w, d_t)
    d_params = None
    if is_mlp:
        tic("fields_backward")
        d_params = G.geraf_fields_backward(field, xyz, saved, d_f, d_G, d_a)
        toc("fields_backward")
    return StepResult(loss, d_params, d_sc, P)


def launches_per_step(field) -> int:
    n = LAUNCHES["sample"] + 3 * LAUNCHES["fields"] + LAUNCHES["blend"] + LAUNCHES["render"]
    n += LAUNCHES["filter"] + LAUNCHES["filter_backward"] + LAUNCHES["render_backward"] + LAUNCHES["blend_backward"]
    if isinstance(field, G.MLPField):
        n += fields_backward_launches(field.n_hidden)
    return n


def terms_per_step(geo: Geometry, n_pts: int) -> int:
    """Phasor terms (point or voxel) x antenna x frequency of the four sums."""
    n_ant = geo.ant.shape[1]
    n_vox = geo.vox.shape[1]
    return 2 * (n_pts + n_vox) * n_ant * geo.band.n_f


def synthetic_target(geo: Geometry, device="cuda") -> torch.Tensor:
    """Heatmap of the analytic sphere (r = 3 cm at 15 cm) + isotropic point
    reflector scene, rendered with uniform samples on the same geometry: the
    synthetic target of the MLP workload."""
    from geraf_inputs import c1_scene
    field = G.AnalyticField(torch.as_tensor(c1_scene().packed(), device=device))
    pr = torch.tensor([[0.0265625], [0.0015625], [0.1203125]], dtype=torch.float32, device=device)
    P, _ = render_heatmap(geo, field, G.SAMPLE_UNIFORM, extra=(pr, torch.ones(1, device=device)))
    return P
