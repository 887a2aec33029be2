"""Thin Python binding of the C ABI (``include/geraf.h``), same call names.

Argument marshalling only: torch supplies device memory and the current CUDA
stream; every step of the rendering path runs in ``libgeraf.so``. Inputs must
be contiguous FP32 CUDA tensors (complex signals may be complex64). Outputs and
workspaces are allocated here with torch and handed to the C call.
"""
import ctypes
from dataclasses import dataclass
from typing import Optional, Sequence

import torch

from . import _lib
from ._lib import GerafBand, GerafFieldDesc, GerafGrid, GerafProposal, check

SAMPLE_UNIFORM, SAMPLE_STRATIFIED = 0, 1
FIELD_ANALYTIC, FIELD_MLP = 0, 1
PREC_FP32, PREC_BF16 = 0, 1
RENDER_DIRECTIONAL = 1
PHASOR_AUTO, PHASOR_RECURRENCE, PHASOR_CHEBYSHEV = 0, 1, 2


def _p(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _req(t: torch.Tensor, name: str, dtype=torch.float32):
    if t is None:
        raise ValueError(f"{name} is required")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (no CPU path)")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _sig(t: torch.Tensor, name: str) -> torch.Tensor:
    """complex64 [n_ant, n_f] or float32 [n_ant, n_f, 2] -> float32 view."""
    if t.dtype == torch.complex64:
        t = torch.view_as_real(t)
    return _req(t, name)


def _alloc_ws(nbytes: int, device) -> torch.Tensor:
    buf = torch.empty(max(int(nbytes), 1) + 256, dtype=torch.uint8, device=device)
    off = (-buf.data_ptr()) % 256
    return buf[off:off + max(int(nbytes), 1)]


def _workspace(fn, device):
    """Runs fn(ws_ptr, ws_bytes_ptr) as a size query, then allocates."""
    n = ctypes.c_size_t(0)
    check(fn(None, ctypes.byref(n)))
    ws = _alloc_ws(n.value, device)
    return ws, ctypes.c_size_t(n.value)


@dataclass
class Band:
    f0: float
    df: float
    n_f: int
    method: int = 0          # PHASOR_AUTO / PHASOR_RECURRENCE / PHASOR_CHEBYSHEV

    def c(self):
        return GerafBand(float(self.f0), float(self.df), int(self.n_f), int(self.method))


def make_grid(lo: Sequence[float], pitch: Sequence[float], n: Sequence[int], aperture_z: float = 0.0) -> GerafGrid:
    g = GerafGrid()
    for d in range(3):
        g.lo[d] = float(lo[d]); g.pitch[d] = float(pitch[d]); g.n[d] = int(n[d])
    g.aperture_z = float(aperture_z)
    return g


class AnalyticField:
    """Scene of analytic primitives: FP32 records [n, 8] = kind, a, c[3], p[3]."""

    def __init__(self, prims: torch.Tensor):
        self.prims = _req(prims.reshape(-1, 8).contiguous(), "prims")

    def desc(self) -> GerafFieldDesc:
        d = GerafFieldDesc()
        d.kind = FIELD_ANALYTIC
        d.prims = self.prims.data_ptr()
        d.n_prims = self.prims.shape[0]
        return d


class MLPField:
    """SDF + reflectiveness MLP with packed FP32 parameters: one trunk with
    head [f, a_logit] (refl_hidden = 0), or the paper's separate SDF and
    reflectivity networks (refl_hidden layers of refl_width for the latter),
    params packed [SDF network | reflectivity network]."""

    def __init__(self, params: torch.Tensor, n_levels=6, width=128, n_hidden=4, beta=100.0,
                 center=(0.0, 0.0, 0.15), half=0.05, precision=PREC_FP32, refl_hidden=0, refl_width=0):
        self.params = _req(params, "params")
        self.n_levels, self.width, self.n_hidden = n_levels, width, n_hidden
        self.beta, self.center, self.half, self.precision = beta, tuple(center), half, precision
        self.refl_hidden, self.refl_width = refl_hidden, refl_width

    @property
    def layer_by_layer(self) -> bool:
        """Networks other than one 128-wide trunk keep their layer activations
        in `saved`, which the library then needs on every call."""
        return self.refl_hidden > 0 or self.width != 128

    def desc(self) -> GerafFieldDesc:
        d = GerafFieldDesc()
        d.kind = FIELD_MLP
        d.params = self.params.data_ptr()
        d.n_levels, d.width, d.n_hidden = self.n_levels, self.width, self.n_hidden
        d.beta = float(self.beta)
        for k in range(3):
            d.center[k] = float(self.center[k])
        d.half = float(self.half)
        d.precision = int(self.precision)
        d.refl_hidden, d.refl_width = int(self.refl_hidden), int(self.refl_width)
        return d


def geraf_check_bounded_wait(limit_ns: int):
    """Self-test of the bounded-wait failure path (see include/geraf.h): the
    next geraf_poll_device_error() raises GerafError with GERAF_ERR_TIMEOUT."""
    check(_lib.lib().geraf_check_bounded_wait(int(limit_ns), _stream()))


def geraf_poll_device_error():
    check(_lib.lib().geraf_poll_device_error(_stream()))


def geraf_sample(grid: GerafGrid, mode: int, seed: int = 0, step: int = 0, device="cuda"):
    """Lensless sampling -> (xyz [3, n_pts], xyz_apr [3, n_ray])."""
    n_ray = grid.n[0] * grid.n[1]
    n = n_ray * grid.n[2]
    xyz = torch.empty(3, n, dtype=torch.float32, device=device)
    apr = torch.empty(3, n_ray, dtype=torch.float32, device=device)
    check(_lib.lib().geraf_sample(ctypes.byref(grid), int(mode), int(seed), int(step), _p(xyz), _p(apr),
                                  _stream()))
    return xyz, apr


def geraf_fields(field, xyz: torch.Tensor, want_grad=True, want_refl=True, keep_saved=False):
    """Fields at points -> (sdf [n], grad [3, n] | None, refl [n] | None, saved | None)."""
    _req(xyz, "xyz")
    n = xyz.shape[-1]
    dev = xyz.device
    desc = field.desc()
    sdf = torch.empty(n, dtype=torch.float32, device=dev)
    grad = torch.empty(3, n, dtype=torch.float32, device=dev) if want_grad else None
    refl = torch.empty(n, dtype=torch.float32, device=dev) if want_refl else None
    saved, nbytes = None, 0
    if keep_saved or getattr(field, "layer_by_layer", False):
        sz = ctypes.c_size_t(0)
        check(_lib.lib().geraf_fields_saved_bytes(ctypes.byref(desc), n, ctypes.byref(sz)))
        nbytes = sz.value
        saved = _alloc_ws(nbytes, dev)
    check(_lib.lib().geraf_fields(ctypes.byref(desc), _p(xyz), n, _p(sdf), _p(grad), _p(refl), _p(saved),
                                  nbytes, _stream()))
    return sdf, grad, refl, saved


def geraf_fields_backward(field, xyz, saved, d_sdf=None, d_grad=None, d_refl=None):
    """Parameter gradient of the MLP fields (same packed layout as params)."""
    _req(xyz, "xyz")
    n = xyz.shape[-1]
    desc = field.desc()
    d_params = torch.empty_like(field.params)
    L = _lib.lib()
    ws, wsz = _workspace(lambda w, b: L.geraf_fields_backward(ctypes.byref(desc), _p(xyz), n, _p(saved),
                                                              _p(d_sdf), _p(d_grad), _p(d_refl), _p(d_params),
                                                              w, b, _stream()), xyz.device)
    check(L.geraf_fields_backward(ctypes.byref(desc), _p(xyz), n, _p(saved), _p(d_sdf), _p(d_grad), _p(d_refl),
                                  _p(d_params), _p(ws), ctypes.byref(wsz), _stream()))
    return d_params


def geraf_blend(sdf, refl, n_ray: int, n_z: int, sdf_apr, sdf_ant, s: float, a_tx: float, keep=None):
    """Lensless alpha blending -> (alpha, T, w, t_eff, c_ant); `keep` (optional,
    per sample) multiplies w, as for the padding samples of geraf_sample_cells."""
    for t, nm in ((sdf, "sdf"), (refl, "refl"), (sdf_apr, "sdf_apr"), (sdf_ant, "sdf_ant")):
        _req(t, nm)
    if keep is not None:
        _req(keep, "keep")
    n = n_ray * n_z
    dev = sdf.device
    alpha, T, w, t_eff = (torch.empty(n, dtype=torch.float32, device=dev) for _ in range(4))
    c_ant = torch.empty(sdf_ant.numel(), dtype=torch.float32, device=dev)
    check(_lib.lib().geraf_blend(_p(sdf), _p(refl), n_ray, n_z, _p(sdf_apr), _p(sdf_ant), sdf_ant.numel(),
                                 float(s), float(a_tx), _p(alpha), _p(T), _p(w), _p(t_eff), _p(c_ant),
                                 _p(keep), _stream()))
    return alpha, T, w, t_eff, c_ant


def geraf_blend_backward(sdf, refl, alpha, T, n_ray, n_z, s, a_tx, d_w=None, d_teff=None, keep=None):
    """-> (d_sdf, d_refl, d_scalars [2] = (dL/ds, dL/dA'_tx)); `keep` as in geraf_blend."""
    n = n_ray * n_z
    dev = sdf.device
    d_sdf = torch.empty(n, dtype=torch.float32, device=dev)
    d_refl = torch.empty(n, dtype=torch.float32, device=dev)
    d_sc = torch.empty(2, dtype=torch.float32, device=dev)
    L = _lib.lib()
    args = lambda w, b: L.geraf_blend_backward(_p(sdf), _p(refl), _p(alpha), _p(T), n_ray, n_z, float(s),
                                               float(a_tx), _p(d_w), _p(d_teff), _p(d_sdf), _p(d_refl), _p(d_sc),
                                               _p(keep), w, b, _stream())
    ws, wsz = _workspace(args, dev)
    check(args(_p(ws), ctypes.byref(wsz)))
    return d_sdf, d_refl, d_sc


def geraf_render(xyz, grad, w, t_eff, ant, c_ant, band: Band, directional=True):
    """Signal tracing -> s complex64 [n_ant, n_f]."""
    for t, nm in ((xyz, "xyz"), (grad, "grad"), (w, "w"), (t_eff, "t_eff"), (ant, "ant"), (c_ant, "c_ant")):
        _req(t, nm)
    n_pts, n_ant = xyz.shape[-1], ant.shape[-1]
    out = torch.empty(n_ant, band.n_f, 2, dtype=torch.float32, device=xyz.device)
    cb = band.c()
    flags = RENDER_DIRECTIONAL if directional else 0
    L = _lib.lib()
    args = lambda wsp, b: L.geraf_render(_p(xyz), _p(grad), _p(w), _p(t_eff), n_pts, _p(ant), _p(c_ant), n_ant,
                                         ctypes.byref(cb), flags, wsp, b, _p(out), _stream())
    ws, wsz = _workspace(args, xyz.device)
    check(args(_p(ws), ctypes.byref(wsz)))
    return torch.view_as_complex(out)


def geraf_render_noalloc(xyz, grad, w, t_eff, ant, c_ant, band: Band, directional=True):
    """Signal tracing without a workspace (the library's static scratch); only
    the output is allocated here. For callers that must not allocate device
    scratch per call; see include/geraf.h for the size limit and the rule that
    overlapping calls race."""
    for t, nm in ((xyz, "xyz"), (grad, "grad"), (w, "w"), (t_eff, "t_eff"), (ant, "ant"), (c_ant, "c_ant")):
        _req(t, nm)
    n_pts, n_ant = xyz.shape[-1], ant.shape[-1]
    out = torch.empty(n_ant, band.n_f, 2, dtype=torch.float32, device=xyz.device)
    cb = band.c()
    check(_lib.lib().geraf_render_noalloc(_p(xyz), _p(grad), _p(w), _p(t_eff), n_pts, _p(ant), _p(c_ant), n_ant,
                                          ctypes.byref(cb), RENDER_DIRECTIONAL if directional else 0, _p(out),
                                          _stream()))
    return torch.view_as_complex(out)


def geraf_render_backward(xyz, grad, w, t_eff, ant, c_ant, band: Band, g_s, directional=True):
    """Adjoint of render -> (d_w [n], d_teff [n], d_grad [3, n])."""
    g = _sig(g_s, "g_s")
    n_pts, n_ant = xyz.shape[-1], ant.shape[-1]
    dev = xyz.device
    d_w = torch.empty(n_pts, dtype=torch.float32, device=dev)
    d_t = torch.empty(n_pts, dtype=torch.float32, device=dev)
    d_g = torch.empty(3, n_pts, dtype=torch.float32, device=dev)
    cb = band.c()
    flags = RENDER_DIRECTIONAL if directional else 0
    L = _lib.lib()
    args = lambda wsp, b: L.geraf_render_backward(_p(xyz), _p(grad), _p(w), _p(t_eff), n_pts, _p(ant), _p(c_ant),
                                                  n_ant, ctypes.byref(cb), flags, _p(g), wsp, b, _p(d_w), _p(d_t),
                                                  _p(d_g), _stream())
    ws, wsz = _workspace(args, dev)
    check(args(_p(ws), ctypes.byref(wsz)))
    return d_w, d_t, d_g


def geraf_filter(s, ant, band: Band, vox, target=None, mask=None):
    """Matched filter -> (P [n_vox], M complex64 [n_vox], loss (0-d float64) | None, dloss_dP | None)."""
    sr = _sig(s, "s")
    _req(ant, "ant"); _req(vox, "vox")
    n_vox, n_ant = vox.shape[-1], ant.shape[-1]
    dev = vox.device
    P = torch.empty(n_vox, dtype=torch.float32, device=dev)
    M = torch.empty(n_vox, 2, dtype=torch.float32, device=dev)
    loss = dP = None
    if target is not None:
        _req(target, "target")
        loss = torch.empty((), dtype=torch.float64, device=dev)
        dP = torch.empty(n_vox, dtype=torch.float32, device=dev)
    if mask is not None:
        _req(mask, "mask")
    cb = band.c()
    L = _lib.lib()
    args = lambda wsp, b: L.geraf_filter(_p(sr), _p(ant), n_ant, ctypes.byref(cb), _p(vox), n_vox, _p(target),
                                         _p(mask), wsp, b, _p(P), _p(M), _p(loss), _p(dP), _stream())
    ws, wsz = _workspace(args, dev)
    check(args(_p(ws), ctypes.byref(wsz)))
    return P, torch.view_as_complex(M), loss, dP


def geraf_masked_loss(P, target, history, t_hi: float, t_lo: float):
    """Dynamic loss masking + masked L2 loss; `history` (running max of P) is
    updated in place. -> (loss 0-d float64, dloss_dP [n], mask [n])."""
    _req(P, "P"); _req(target, "target"); _req(history, "history")
    n = P.shape[-1]
    dev = P.device
    loss = torch.empty((), dtype=torch.float64, device=dev)
    dP = torch.empty(n, dtype=torch.float32, device=dev)
    mask = torch.empty(n, dtype=torch.float32, device=dev)
    L = _lib.lib()
    args = lambda wsp, b: L.geraf_masked_loss(_p(P), _p(target), _p(history), n, float(t_hi), float(t_lo), wsp, b,
                                              _p(loss), _p(dP), _p(mask), _stream())
    ws, wsz = _workspace(args, dev)
    check(args(_p(ws), ctypes.byref(wsz)))
    return loss, dP, mask


def geraf_filter_backward(ant, band: Band, vox, M, d_P):
    """Adjoint of |matched filter| -> g_s complex64 [n_ant, n_f]."""
    Mr = _sig(M, "M")
    _req(d_P, "d_P")
    n_vox, n_ant = vox.shape[-1], ant.shape[-1]
    out = torch.empty(n_ant, band.n_f, 2, dtype=torch.float32, device=vox.device)
    cb = band.c()
    L = _lib.lib()
    args = lambda wsp, b: L.geraf_filter_backward(_p(ant), n_ant, ctypes.byref(cb), _p(vox), n_vox, _p(Mr),
                                                  _p(d_P), wsp, b, _p(out), _stream())
    ws, wsz = _workspace(args, vox.device)
    check(args(_p(ws), ctypes.byref(wsz)))
    return torch.view_as_complex(out)


def geraf_chebyshev_order(xyz, ant, band: Band) -> int:
    """Chebyshev order the phasor sums use for these points and antennas
    (0: the per-bin recurrence runs). Synchronous."""
    _req(xyz, "xyz")
    _req(ant, "ant")
    cb = band.c()
    order = ctypes.c_int32(-1)
    L = _lib.lib()
    args = lambda wsp, b: L.geraf_chebyshev_order(_p(xyz), xyz.shape[-1], _p(ant), ant.shape[-1], ctypes.byref(cb),
                                                  wsp, b, ctypes.byref(order), _stream())
    ws, wsz = _workspace(args, xyz.device)
    check(args(_p(ws), ctypes.byref(wsz)))
    return int(order.value)


def geraf_chebyshev_work(xyz, ant, band: Band, to_points: bool):
    """Orders one Chebyshev phasor call evaluates: (K of the whole set, the
    largest split or group order, the kernel instance's compiled orders, the
    mean orders evaluated per (point, antenna) pair). to_points: the
    direction of geraf_filter / geraf_render_backward, else that of
    geraf_render / geraf_filter_backward. All zero when the recurrence runs.
    Synchronous."""
    _req(xyz, "xyz")
    _req(ant, "ant")
    cb = band.c()
    orders = (ctypes.c_int32 * 3)()
    mean = ctypes.c_double(0.0)
    L = _lib.lib()
    args = lambda wsp, b: L.geraf_chebyshev_work(_p(xyz), xyz.shape[-1], _p(ant), ant.shape[-1], ctypes.byref(cb),
                                                 1 if to_points else 0, wsp, b, orders, ctypes.byref(mean),
                                                 _stream())
    ws, wsz = _workspace(args, xyz.device)
    check(args(_p(ws), ctypes.byref(wsz)))
    return int(orders[0]), int(orders[1]), int(orders[2]), float(mean.value)


class Proposal:
    """Learned proposal: FP16 feature grid [G2, G1, G0, feat] and FP32 MLP params."""

    def __init__(self, features: torch.Tensor, params: torch.Tensor, width=64, n_hidden=3, beta=10.0, eps=0.01,
                 depth=16):
        if features.dtype != torch.float16 or features.dim() != 4:
            raise ValueError("features must be float16 [G2, G1, G0, feat]")
        self.features = _req(features, "features", torch.float16)
        self.params = _req(params, "params")
        self.width, self.n_hidden, self.beta, self.eps, self.depth = width, n_hidden, beta, eps, depth

    @property
    def gshape(self):
        G2, G1, G0, _ = self.features.shape
        return (G0, G1, G2)

    @property
    def n_cells(self):
        return self.features.shape[0] * self.features.shape[1] * self.features.shape[2]

    def c(self) -> GerafProposal:
        p = GerafProposal()
        p.features = self.features.data_ptr()
        p.params = self.params.data_ptr()
        G0, G1, G2 = self.gshape
        p.g[0], p.g[1], p.g[2] = G0, G1, G2
        p.feat = self.features.shape[3]
        p.width, p.n_hidden, p.beta, p.eps, p.depth = self.width, self.n_hidden, float(self.beta), float(self.eps), \
            self.depth
        return p


def geraf_proposal_density(prop: Proposal, keep_saved=True):
    """-> (logits [n_cells], q [n_cells], saved | None), cells ordered (gz, gy, gx)."""
    dev = prop.features.device
    cp = prop.c()
    logits = torch.empty(prop.n_cells, dtype=torch.float32, device=dev)
    q = torch.empty(prop.n_cells, dtype=torch.float32, device=dev)
    saved, nbytes = None, 0
    if keep_saved:
        sz = ctypes.c_size_t(0)
        check(_lib.lib().geraf_proposal_saved_bytes(ctypes.byref(cp), ctypes.byref(sz)))
        nbytes = sz.value
        saved = _alloc_ws(nbytes, dev)
    check(_lib.lib().geraf_proposal_density(ctypes.byref(cp), _p(logits), _p(q), _p(saved), nbytes, _stream()))
    return logits, q, saved


def geraf_sample_proposal(grid: GerafGrid, prop: Proposal, q, seed=0, step=0):
    """-> (xyz [3, n_ray*depth], xyz_apr [3, n_ray], idx int32 [n_ray*depth])."""
    dev = prop.features.device
    n_ray = grid.n[0] * grid.n[1]
    n = n_ray * prop.depth
    xyz = torch.empty(3, n, dtype=torch.float32, device=dev)
    apr = torch.empty(3, n_ray, dtype=torch.float32, device=dev)
    idx = torch.empty(n, dtype=torch.int32, device=dev)
    cp = prop.c()
    check(_lib.lib().geraf_sample_proposal(ctypes.byref(grid), ctypes.byref(cp), _p(_req(q, "q")), int(seed),
                                           int(step), _p(xyz), _p(apr), _p(idx), _stream()))
    return xyz, apr, idx


def geraf_sample_cells(grid: GerafGrid, prop: Proposal, q, m: int, r_max: int, seed=0, step=0, dilate=0):
    """Stratified grid samples of the m proposal cells of largest q per column,
    with run-closing samples -> (xyz [3, n_ray*n_out], xyz_apr [3, n_ray],
    idx int32 [n_ray*n_out], keep [n_ray*n_out], n_out = m s + r_max)."""
    dev = prop.features.device
    n_ray = grid.n[0] * grid.n[1]
    s_fine = grid.n[2] // prop.gshape[2]
    n_out = m * s_fine + r_max
    n = n_ray * n_out
    xyz = torch.empty(3, n, dtype=torch.float32, device=dev)
    apr = torch.empty(3, n_ray, dtype=torch.float32, device=dev)
    idx = torch.empty(n, dtype=torch.int32, device=dev)
    keep = torch.empty(n, dtype=torch.float32, device=dev)
    cp = prop.c()
    L = _lib.lib()
    args = lambda w, b: L.geraf_sample_cells(ctypes.byref(grid), ctypes.byref(cp), _p(_req(q, "q")), int(m),
                                             int(r_max), int(dilate), int(seed), int(step), _p(xyz), _p(apr), _p(idx),
                                             _p(keep), w, b, _stream())
    ws, wsz = _workspace(args, dev)
    check(args(_p(ws), ctypes.byref(wsz)))
    return xyz, apr, idx, keep, n_out


def geraf_sample_backward(prop: Proposal, grid: GerafGrid, n_z: int, alpha, T, idx, logits, saved):
    """-> (d_params, d_features FP32 [G2, G1, G0, feat], loss 0-d float64)."""
    dev = prop.features.device
    cp = prop.c()
    d_params = torch.empty_like(prop.params)
    d_feat = torch.empty(prop.features.shape, dtype=torch.float32, device=dev)
    loss = torch.empty((), dtype=torch.float64, device=dev)
    L = _lib.lib()
    args = lambda w, b: L.geraf_sample_backward(ctypes.byref(cp), ctypes.byref(grid), int(n_z), _p(alpha), _p(T),
                                                _p(idx), _p(logits), _p(saved), _p(d_params), _p(d_feat), _p(loss),
                                                w, b, _stream())
    ws, wsz = _workspace(args, dev)
    check(args(_p(ws), ctypes.byref(wsz)))
    return d_params, d_feat, loss
