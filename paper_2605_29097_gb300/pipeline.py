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
# with the Chebyshev form each phasor call launches: the whole-call range bound
# and plan (2), the points' brick-order sort (4), the antenna order (2), the
# record packs, the part bounds and plans, three kernel instances (those that
# do not apply return at once), the to-bins reconstruction and split-group sum
# or the to-points antenna rows, and the recurrence kernels and their
# reduction (launched either way; they return at once unless the device-side
# plan falls back to them): 19 per call, counted from the launch list of one
# step of the 256^3-sample workload (90 launches per step with the 4x128 network)
LAUNCHES_CHEBYSHEV = {"render": 19, "filter": 19, "filter_backward": 19, "render_backward": 19}


def uses_chebyshev(band) -> bool:
    if band.method == G.PHASOR_RECURRENCE:
        return False
    return band.method == G.PHASOR_CHEBYSHEV or band.n_f >= 64


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


class DynamicMask:
    """State of the dynamic loss masking (section 6): the running maximum of
    each voxel's rendered power over earlier steps, and the two thresholds,
    taken relative to the target's maximum (the paper gives no values): high
    = rho_hi * max(target), low = rho_lo * max(target)."""

    def __init__(self, target: torch.Tensor, rho_hi=0.5, rho_lo=0.1):
        p_ref = float(target.max())
        self.t_hi = float(np.float32(rho_hi * p_ref))
        self.t_lo = float(np.float32(rho_lo * p_ref))
        self.history = torch.zeros_like(target)


def forward_backward(geo: Geometry, field, target: torch.Tensor, seed: int, step: int, timers=None,
                     dyn_mask: Optional[DynamicMask] = None) -> StepResult:
    """One hot-path pass (all forward steps and their adjoints). `timers` may map
    a step name to a pair of CUDA events recorded around that call; with
    `dyn_mask` the loss leaves out the voxels the dynamic mask drops."""
    def tic(name):
        if timers is not None and name in timers:
            timers[name][0].record()

    def toc(name):
        if timers is not None and name in timers:
            timers[name][1].record()

    xyz, apr = G.geraf_sample(geo.grid, geo.mode, seed, step, device=geo.ant.device)
    is_mlp = isinstance(field, G.MLPField)
    tic("fields")
    f, grad, a, saved = G.geraf_fields(field, xyz, keep_saved=is_mlp)
    toc("fields")
    fa, _, _, _ = G.geraf_fields(field, apr, want_grad=False, want_refl=False)
    fn, _, _, _ = G.geraf_fields(field, geo.ant, want_grad=False, want_refl=False)
    alpha, T, w, t_eff, c_ant = G.geraf_blend(f, a, geo.n_ray, geo.n_z, fa, fn, geo.sharpness, geo.a_tx)
    tic("render")
    s = G.geraf_render(xyz, grad, w, t_eff, geo.ant, c_ant, geo.band)
    toc("render")
    tic("filter")
    mask = None
    if dyn_mask is None:
        P, M, loss, dP = G.geraf_filter(s, geo.ant, geo.band, geo.vox, target)
    else:
        P, M, _, _ = G.geraf_filter(s, geo.ant, geo.band, geo.vox)
        loss, dP, mask = G.geraf_masked_loss(P, target, dyn_mask.history, dyn_mask.t_hi, dyn_mask.t_lo)
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
    res = StepResult(loss, d_params, d_sc, P)
    res.mask = mask
    return res


def launches_per_step(field, band) -> int:
    ph = LAUNCHES_CHEBYSHEV if uses_chebyshev(band) else LAUNCHES
    n = LAUNCHES["sample"] + 3 * LAUNCHES["fields"] + LAUNCHES["blend"] + LAUNCHES["blend_backward"]
    n += ph["render"] + ph["filter"] + ph["filter_backward"] + ph["render_backward"]
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


# ------------------------------------------------------------- training step
def scene_field(scene, device="cuda"):
    return G.AnalyticField(torch.as_tensor(scene.packed(), device=device))


def scene_signal(geo: Geometry, scene, occluder_z=None, atten=1.0, mode=G.SAMPLE_UNIFORM, seed=0, device="cuda"):
    """Clean signal of an analytic scene; points beyond the occluder plane get
    the round-trip amplitude factor `atten` (set-up only: torch scales w)."""
    field = scene_field(scene, device)
    xyz, apr = G.geraf_sample(geo.grid, mode, seed, 0, device=device)
    f, grad, a, _ = G.geraf_fields(field, xyz)
    fa, _, _, _ = G.geraf_fields(field, apr, want_grad=False, want_refl=False)
    fn, _, _, _ = G.geraf_fields(field, geo.ant, want_grad=False, want_refl=False)
    _, _, w, t_eff, c_ant = G.geraf_blend(f, a, geo.n_ray, geo.n_z, fa, fn, geo.sharpness, geo.a_tx)
    if occluder_z is not None:
        w = torch.where(xyz[2] > occluder_z, w * atten, w).contiguous()
    return G.geraf_render(xyz, grad, w, t_eff, geo.ant, c_ant, geo.band)


def scene_target(geo: Geometry, scene, noise_seed=0, device="cuda"):
    """Synthetic target of the training workload: analytic scene behind a
    0.5-attenuation occluder plane, complex Gaussian noise at 10 dB SNR on the
    signal, matched-filtered on the heatmap voxels."""
    import geraf_inputs as gi
    s = scene_signal(geo, scene, gi.C4_OCCLUDER_Z, gi.C4_OCCLUDER_ATTEN, device=device)
    power = float((s.abs() ** 2).mean())
    noise = torch.as_tensor(gi.c4_noise(noise_seed, tuple(s.shape), power).astype(np.complex64), device=device)
    P, _, _, _ = G.geraf_filter((s + noise).contiguous(), geo.ant, geo.band, geo.vox)
    return P


def geometry_with_depths(geo: Geometry, n_z: int) -> Geometry:
    """Same columns, cube and radar with n_z depth cells per column."""
    g = G.make_grid([geo.grid.lo[d] for d in range(3)],
                    [geo.grid.pitch[0], geo.grid.pitch[1], geo.grid.pitch[2] * geo.grid.n[2] / n_z],
                    [geo.grid.n[0], geo.grid.n[1], n_z], geo.grid.aperture_z)
    return Geometry(g, geo.n_ray, n_z, geo.ant, geo.vox, geo.band, geo.sharpness, geo.a_tx, geo.mode)


def proposal_forward_backward(geo: Geometry, field, prop, target, seed: int, step: int, timers=None):
    """One hot-path pass with depths drawn from the learned proposal (depth
    samples per column = prop.depth), plus the proposal's own training signal
    from the blended weights of this pass."""
    def tic(name):
        if timers is not None and name in timers:
            timers[name][0].record()

    def toc(name):
        if timers is not None and name in timers:
            timers[name][1].record()

    logits, q, psaved = G.geraf_proposal_density(prop)
    xyz, apr, idx = G.geraf_sample_proposal(geo.grid, prop, q, seed, step)
    n_z = prop.depth
    is_mlp = isinstance(field, G.MLPField)
    f, grad, a, saved = G.geraf_fields(field, xyz, keep_saved=is_mlp)
    fa, _, _, _ = G.geraf_fields(field, apr, want_grad=False, want_refl=False)
    fn, _, _, _ = G.geraf_fields(field, geo.ant, want_grad=False, want_refl=False)
    alpha, T, w, t_eff, c_ant = G.geraf_blend(f, a, geo.n_ray, n_z, fa, fn, geo.sharpness, geo.a_tx)
    tic("render")
    s = G.geraf_render(xyz, grad, w, t_eff, geo.ant, c_ant, geo.band)
    toc("render")
    P, M, loss, dP = G.geraf_filter(s, geo.ant, geo.band, geo.vox, target)
    g_s = G.geraf_filter_backward(geo.ant, geo.band, geo.vox, M, dP)
    tic("render_backward")
    d_w, d_t, d_G = G.geraf_render_backward(xyz, grad, w, t_eff, geo.ant, c_ant, geo.band, g_s)
    toc("render_backward")
    d_f, d_a, d_sc = G.geraf_blend_backward(f, a, alpha, T, geo.n_ray, n_z, geo.sharpness, geo.a_tx, d_w, d_t)
    d_params = G.geraf_fields_backward(field, xyz, saved, d_f, d_G, d_a) if is_mlp else None
    dp_prop, df_prop, ploss = G.geraf_sample_backward(prop, geo.grid, n_z, alpha, T, idx, logits, psaved)
    res = StepResult(loss, d_params, d_sc, P)
    res.proposal = (dp_prop, df_prop, ploss)
    return res


def cells_forward_backward(geo: Geometry, field, prop, target, m: int, r_max: int, seed: int, step: int,
                           q=None, timers=None, train_proposal=True, dilate=1):
    """One hot-path pass on the stratified grid's own samples in the m proposal
    cells of largest q per column (geraf_sample_cells: closing samples after
    each run, keep = 0 on closing and padding samples), plus the proposal's
    training signal from this pass's blended weights. `q` overrides the
    proposal's own distribution (for measurements)."""
    def tic(name):
        if timers is not None and name in timers:
            timers[name][0].record()

    def toc(name):
        if timers is not None and name in timers:
            timers[name][1].record()

    logits, q_prop, psaved = G.geraf_proposal_density(prop)
    xyz, apr, idx, keep, n_out = G.geraf_sample_cells(geo.grid, prop, q_prop if q is None else q, m, r_max, seed,
                                                      step, dilate=dilate)
    is_mlp = isinstance(field, G.MLPField)
    f, grad, a, saved = G.geraf_fields(field, xyz, keep_saved=is_mlp)
    fa, _, _, _ = G.geraf_fields(field, apr, want_grad=False, want_refl=False)
    fn, _, _, _ = G.geraf_fields(field, geo.ant, want_grad=False, want_refl=False)
    alpha, T, w, t_eff, c_ant = G.geraf_blend(f, a, geo.n_ray, n_out, fa, fn, geo.sharpness, geo.a_tx, keep)
    tic("render")
    s = G.geraf_render(xyz, grad, w, t_eff, geo.ant, c_ant, geo.band)
    toc("render")
    P, M, loss, dP = G.geraf_filter(s, geo.ant, geo.band, geo.vox, target)
    g_s = G.geraf_filter_backward(geo.ant, geo.band, geo.vox, M, dP)
    tic("render_backward")
    d_w, d_t, d_G = G.geraf_render_backward(xyz, grad, w, t_eff, geo.ant, c_ant, geo.band, g_s)
    toc("render_backward")
    d_f, d_a, d_sc = G.geraf_blend_backward(f, a, alpha, T, geo.n_ray, n_out, geo.sharpness, geo.a_tx, d_w, d_t,
                                            keep)
    d_params = G.geraf_fields_backward(field, xyz, saved, d_f, d_G, d_a) if is_mlp else None
    res = StepResult(loss, d_params, d_sc, P)
    res.n_out = n_out
    res.proposal = (G.geraf_sample_backward(prop, geo.grid, n_out, alpha, T, idx, logits, psaved)
                    if train_proposal else None)
    return res


def dense_weight_histogram(geo: Geometry, field, gshape, seed: int, step: int):
    """Measurement helper: per proposal grid column, the normalised histogram
    of the dense stratified render's geometric weights T alpha over its G2
    depth cells (fine columns of a grid column pooled), as FP32 q [n_cells]
    ordered (gz, gy, gx): the distribution a perfect proposal would learn."""
    G0, G1, G2 = gshape
    xyz, apr = G.geraf_sample(geo.grid, geo.mode, seed, step, device=geo.ant.device)
    f, _, a, _ = G.geraf_fields(field, xyz, want_grad=False)
    fa, _, _, _ = G.geraf_fields(field, apr, want_grad=False, want_refl=False)
    fn, _, _, _ = G.geraf_fields(field, geo.ant, want_grad=False, want_refl=False)
    alpha, T, _, _, _ = G.geraf_blend(f, a, geo.n_ray, geo.n_z, fa, fn, geo.sharpness, geo.a_tx)
    nx, ny, nz = geo.grid.n[0], geo.grid.n[1], geo.grid.n[2]
    # depth-major [nz][ny][nx] -> [cell z, fine z, grid y, fine y, grid x, fine x], summed over the fine axes
    h = (T * alpha).double().view(G2, nz // G2, G1, ny // G1, G0, nx // G0).sum(dim=(1, 3, 5))
    h = h / h.sum(dim=0, keepdim=True).clamp_min(1e-300)
    return h.float().contiguous().reshape(-1)


def proposal_signal_dense(geo: Geometry, field, prop, seed: int, step: int):
    """Proposal training signal from a dense regular-grid render of `field`
    (geo.grid's own depths, a multiple of the proposal's G2)."""
    logits, q, psaved = G.geraf_proposal_density(prop)
    xyz, apr = G.geraf_sample(geo.grid, geo.mode, seed, step, device=geo.ant.device)
    f, _, a, _ = G.geraf_fields(field, xyz, want_grad=False)
    fa, _, _, _ = G.geraf_fields(field, apr, want_grad=False, want_refl=False)
    fn, _, _, _ = G.geraf_fields(field, geo.ant, want_grad=False, want_refl=False)
    alpha, T, _, _, _ = G.geraf_blend(f, a, geo.n_ray, geo.n_z, fa, fn, geo.sharpness, geo.a_tx)
    return G.geraf_sample_backward(prop, geo.grid, geo.n_z, alpha, T, None, logits, psaved)


def proposal_heatmap(geo: Geometry, field, prop, seed=0, step=0):
    """Forward-only heatmap with proposal-drawn depths."""
    _, q, _ = G.geraf_proposal_density(prop, keep_saved=False)
    xyz, apr, _ = G.geraf_sample_proposal(geo.grid, prop, q, seed, step)
    f, grad, a, _ = G.geraf_fields(field, xyz)
    fa, _, _, _ = G.geraf_fields(field, apr, want_grad=False, want_refl=False)
    fn, _, _, _ = G.geraf_fields(field, geo.ant, want_grad=False, want_refl=False)
    _, _, w, t_eff, c_ant = G.geraf_blend(f, a, geo.n_ray, prop.depth, fa, fn, geo.sharpness, geo.a_tx)
    s = G.geraf_render(xyz, grad, w, t_eff, geo.ant, c_ant, geo.band)
    P, _, _, _ = G.geraf_filter(s, geo.ant, geo.band, geo.vox)
    return P


def init_proposal(gshape=(64, 64, 64), feat=8, width=64, n_hidden=3, depth=16, seed=0, eps=0.01, device="cuda"):
    """Seeded initial proposal (small random features, U(+-1/sqrt(fan_in)) MLP)."""
    G0, G1, G2 = gshape
    rng = np.random.default_rng(seed)
    feats = (0.1 * rng.standard_normal((G2, G1, G0, feat))).astype(np.float32)
    shapes = [(width, feat)] + [(width, width)] * (n_hidden - 1) + [(1, width)]
    parts = []
    for o, i in shapes:
        parts += [rng.uniform(-1 / np.sqrt(i), 1 / np.sqrt(i), o * i), np.zeros(o)]
    params = np.concatenate(parts).astype(np.float32)
    master = torch.as_tensor(feats, device=device).requires_grad_(False)
    prop = G.Proposal(master.half(), torch.as_tensor(params, device=device), width=width, n_hidden=n_hidden,
                      eps=eps, depth=depth)
    return prop, master


class ProposalTrainer:
    """AdamW on the proposal (FP32 master features, FP16 copy for the kernels)."""

    def __init__(self, prop, master, lr=1e-2):
        self.prop, self.master = prop, master
        self.params = prop.params.detach().clone().requires_grad_(True)
        self.feats = master.detach().clone().requires_grad_(True)
        self.opt = torch.optim.Adam([self.params, self.feats], lr=lr)

    def step(self, d_params, d_feat):
        self.opt.zero_grad(set_to_none=False)
        self.params.grad = d_params.clone()
        self.feats.grad = d_feat.clone()
        self.opt.step()
        with torch.no_grad():
            self.prop.params.copy_(self.params)
            self.prop.features.copy_(self.feats.half())


# ------------------------------------------------------ signal tracing bank
class SignalBank:
    """Signal tracing bank (section 5.3 "Signal Tracing Bank"): the aperture is
    divided into patches of antennas, each step traces the signal of one patch
    only and takes every other antenna's signal from the bank, which the step
    then updates with the patch it traced. The matched filter has no
    parameters, so bank entries carry no gradient: the filter adjoint and the
    tracing adjoint run for the traced patch alone.

    The antennas are reordered patch by patch (patches are px x py tiles of the
    nx x ny array, patch k = qy * (nx / px) + qx) so that each patch is a
    contiguous range of bank rows; `order[i]` is the original index of bank
    row i and `geo` is the geometry in bank order."""

    def __init__(self, geo: Geometry, array_shape, patch_shape):
        nx, ny = array_shape
        px, py = patch_shape
        if nx * ny != geo.ant.shape[1] or nx % px or ny % py:
            raise ValueError("patch shape must tile the antenna array")
        idx = np.arange(nx * ny).reshape(ny, nx)
        order = np.concatenate([idx[qy * py:(qy + 1) * py, qx * px:(qx + 1) * px].reshape(-1)
                                for qy in range(ny // py) for qx in range(nx // px)])
        self.order = order
        dev = geo.ant.device
        ant = geo.ant[:, torch.as_tensor(order, device=dev)].contiguous()
        self.geo = Geometry(geo.grid, geo.n_ray, geo.n_z, ant, geo.vox, geo.band, geo.sharpness, geo.a_tx, geo.mode)
        self.patch_size = px * py
        self.n_patch = (nx // px) * (ny // py)
        self.patch_ant = [ant[:, k * self.patch_size:(k + 1) * self.patch_size].contiguous()
                          for k in range(self.n_patch)]
        self.s = torch.zeros(nx * ny, geo.band.n_f, dtype=torch.complex64, device=dev)

    def rows(self, k):
        return k * self.patch_size, (k + 1) * self.patch_size

    def fill(self, field, seed: int, step: int):
        """Trace every antenna once (the bank's initial content)."""
        _, s = render_heatmap(self.geo, field, self.geo.mode, seed, step)
        self.s.copy_(s)


def forward_backward_bank(bank: SignalBank, field, target: torch.Tensor, seed: int, step: int, patch=None,
                          timers=None) -> StepResult:
    """One hot-path pass with the signal tracing bank: trace patch `patch`
    (default: step mod the number of patches), update its bank rows, filter
    the whole bank against the target, and run the adjoints for that patch."""
    def tic(name):
        if timers is not None and name in timers:
            timers[name][0].record()

    def toc(name):
        if timers is not None and name in timers:
            timers[name][1].record()

    geo = bank.geo
    k = step % bank.n_patch if patch is None else patch
    a0, a1 = bank.rows(k)
    ant_p = bank.patch_ant[k]
    xyz, apr = G.geraf_sample(geo.grid, geo.mode, seed, step, device=geo.ant.device)
    is_mlp = isinstance(field, G.MLPField)
    f, grad, a, saved = G.geraf_fields(field, xyz, keep_saved=is_mlp)
    fa, _, _, _ = G.geraf_fields(field, apr, want_grad=False, want_refl=False)
    fn, _, _, _ = G.geraf_fields(field, ant_p, want_grad=False, want_refl=False)
    alpha, T, w, t_eff, c_ant = G.geraf_blend(f, a, geo.n_ray, geo.n_z, fa, fn, geo.sharpness, geo.a_tx)
    tic("render")
    s_p = G.geraf_render(xyz, grad, w, t_eff, ant_p, c_ant, geo.band)
    toc("render")
    bank.s[a0:a1].copy_(s_p)
    tic("filter")
    P, M, loss, dP = G.geraf_filter(bank.s, geo.ant, geo.band, geo.vox, target)
    toc("filter")
    tic("filter_backward")
    g_p = G.geraf_filter_backward(ant_p, geo.band, geo.vox, M, dP)
    toc("filter_backward")
    tic("render_backward")
    d_w, d_t, d_G = G.geraf_render_backward(xyz, grad, w, t_eff, ant_p, c_ant, geo.band, g_p)
    toc("render_backward")
    d_f, d_a, d_sc = G.geraf_blend_backward(f, a, alpha, T, geo.n_ray, geo.n_z, geo.sharpness, geo.a_tx, d_w, d_t)
    d_params = None
    if is_mlp:
        tic("fields_backward")
        d_params = G.geraf_fields_backward(field, xyz, saved, d_f, d_G, d_a)
        toc("fields_backward")
    res = StepResult(loss, d_params, d_sc, P)
    res.bank = {"patch": k, "xyz": xyz, "grad": grad, "w": w, "t_eff": t_eff, "c_ant": c_ant, "M": M, "dP": dP,
                "g": g_p, "d_w": d_w, "d_teff": d_t, "d_G": d_G}
    return res


# ------------------------------------------------------ checkpoint / resume
def save_checkpoint(path, step: int, params: torch.Tensor, optimizer=None, proposal=None, proposal_trainer=None,
                    extra=None):
    """Training state to `path` (torch.save): the packed field parameters, the
    optimiser state, the proposal (FP16 features and its MLP, with its own
    trainer's FP32 masters and Adam state) and the step counter. Sampling
    jitter and proposal draws come from counter-based generators keyed by
    (seed, step, index), so resuming at `step` repeats the same samples."""
    state = {"step": int(step), "params": params.detach().cpu()}
    if optimizer is not None:
        state["optimizer"] = optimizer.state_dict()
    if proposal is not None:
        state["proposal"] = {"features": proposal.features.detach().cpu(), "params": proposal.params.detach().cpu()}
    if proposal_trainer is not None:
        state["proposal_trainer"] = {"params": proposal_trainer.params.detach().cpu(),
                                     "feats": proposal_trainer.feats.detach().cpu(),
                                     "optimizer": proposal_trainer.opt.state_dict()}
    if extra is not None:
        state["extra"] = extra
    torch.save(state, path)


def load_checkpoint(path, params: torch.Tensor, optimizer=None, proposal=None, proposal_trainer=None) -> dict:
    """Restores what save_checkpoint wrote into the given tensors and
    optimisers (in place, on their devices); returns the state dict (its
    "step" is the step to continue from)."""
    state = torch.load(path, map_location="cpu", weights_only=False)
    with torch.no_grad():
        params.copy_(state["params"].to(params.device))
    if optimizer is not None and "optimizer" in state:
        optimizer.load_state_dict(state["optimizer"])
    if proposal is not None and "proposal" in state:
        with torch.no_grad():
            proposal.features.copy_(state["proposal"]["features"].to(proposal.features.device))
            proposal.params.copy_(state["proposal"]["params"].to(proposal.params.device))
    if proposal_trainer is not None and "proposal_trainer" in state:
        pt = state["proposal_trainer"]
        with torch.no_grad():
            proposal_trainer.params.copy_(pt["params"].to(proposal_trainer.params.device))
            proposal_trainer.feats.copy_(pt["feats"].to(proposal_trainer.feats.device))
        proposal_trainer.opt.load_state_dict(pt["optimizer"])
    return state
