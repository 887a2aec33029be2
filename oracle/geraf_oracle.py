"""FP64 CPU oracle of GeRaF's lensless, full-space RF volumetric rendering.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import or run this package. It
shares no code with the CUDA product path (``paper_2605_29097_gb300``) and
imports nothing from it; inputs come from ``geraf_inputs`` (set-up only).

Each function states the paper passage it follows. Floating point is FP64
throughout: FP32 inputs are promoted exactly, FP64 results are returned. A
library primitive (numpy matmul, libm cos/sin) may serve as one step; there is
no blocking, fusion or reordering beyond the definitions. The four phasor sums
are plain C loop nests in ``phasor_oracle.c``.

Pins: every function is checked by ``tests/test_oracle_*.py`` against closed
forms, printed paper values, invariants, brute force or an independent library
(torch autograd); none of its parts is "parity unpinned".
"""
import ctypes
import os

import numpy as np

from . import build as _build

C_LIGHT = 299792458.0  # m/s, exact SI value

# --------------------------------------------------------------------------
# Counter-based uniform generator: SplitMix64 (Steele, Lea & Flood, "Fast
# splittable pseudorandom number generators", OOPSLA 2014), output function
# z = state + (k+1)*gamma; z ^= z>>30; z *= C1; z ^= z>>27; z *= C2; z ^= z>>31.
# --------------------------------------------------------------------------
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, k):
    """k-th output (k = 0, 1, ...) of SplitMix64 seeded with ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.asarray(k, dtype=np.uint64) + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _MIX1
        z = (z ^ (z >> np.uint64(27))) * _MIX2
        return z ^ (z >> np.uint64(31))


def uniform01(seed, step, stream, index):
    """U in [0, 1): top 53 bits of SplitMix64 output number
    (step << 42 | stream << 40 | index), scaled by 2^-53 (exact in FP64)."""
    index = np.asarray(index, dtype=np.uint64)
    k = (np.uint64(step) << np.uint64(42)) | (np.uint64(stream) << np.uint64(40)) | index
    return (splitmix64(seed, k) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


# --------------------------------------------------------------------------
# Lensless sampling (section 6 "Primary Ray"): parallel primary rays along the
# radar's primary direction p = +z start at x_apr in the aperture plane;
# points x = x_apr + u p. Full-space grid: column (ix, iy) of the cube face,
# N_z depths; uniform = cell centres, stratified = cell minimum + U * pitch with
# one U per column axis (the ray start) and one per depth (the point).
# --------------------------------------------------------------------------

def _coord(lo, i, frac, pitch):
    """float32( lo + (i + frac) * pitch ), each operation one FP64 rounding."""
    t = np.asarray(i, dtype=np.float64) + frac
    t = t * np.float64(np.float32(pitch))
    return (np.float64(np.float32(lo)) + t).astype(np.float32)


def sample(grid, mode, seed=0, step=0):
    """Returns (xyz [3, N] float32 depth-major, x_apr [3, N_ray] float32)."""
    nx, ny, nz = grid.n
    n_ray = nx * ny
    ray = np.arange(n_ray, dtype=np.int64)
    ix, iy = ray % nx, ray // nx
    pts = np.arange(n_ray * nz, dtype=np.int64)
    k = pts // n_ray
    if mode == 0:
        ux = uy = 0.5
        uz = 0.5
    else:
        ux = uniform01(seed, step, 0, ray)
        uy = uniform01(seed, step, 1, ray)
        uz = uniform01(seed, step, 2, pts)
    xr = _coord(grid.lo[0], ix, ux, grid.pitch[0])
    yr = _coord(grid.lo[1], iy, uy, grid.pitch[1])
    xyz = np.empty((3, n_ray * nz), dtype=np.float32)
    xyz[0] = np.tile(xr, nz)
    xyz[1] = np.tile(yr, nz)
    xyz[2] = _coord(grid.lo[2], k, uz, grid.pitch[2])
    apr = np.empty((3, n_ray), dtype=np.float32)
    apr[0], apr[1], apr[2] = xr, yr, np.float32(grid.aperture_z)
    return xyz, apr


# --------------------------------------------------------------------------
# Analytic fields (SDF f, its gradient G = grad f, reflectiveness a).
# The scene SDF is the minimum over primitives (union); G and a are those of
# the minimising primitive (first one on ties).
# --------------------------------------------------------------------------

def _prim_sdf(kind, c, p, x):
    d = x - np.asarray(c, dtype=np.float64)[:, None]
    if kind == 0:      # sphere |x - c| - R
        r = np.sqrt((d * d).sum(0))
        with np.errstate(invalid="ignore", divide="ignore"):
            G = np.where(r > 0, d / r, 0.0)
        return r - p[0], G
    if kind == 1:      # box with half extents h
        h = np.asarray(p, dtype=np.float64)[:, None]
        q = np.abs(d) - h
        qp = np.maximum(q, 0.0)
        out = np.sqrt((qp * qp).sum(0))
        qmax = q.max(0)
        f = out + np.minimum(qmax, 0.0)
        sgn = np.where(d >= 0, 1.0, -1.0)
        with np.errstate(invalid="ignore", divide="ignore"):
            G_out = sgn * qp / out
        am = q.argmax(0)
        G_in = np.zeros_like(d)
        G_in[am, np.arange(d.shape[1])] = sgn[am, np.arange(d.shape[1])]
        G = np.where(qmax > 0, G_out, G_in)
        return f, G
    if kind == 2:      # ellipsoid, first-order scaled-sphere distance (|d/R| - 1) min R
        R = np.asarray(p, dtype=np.float64)[:, None]
        e = d / R
        k0 = np.sqrt((e * e).sum(0))
        m = R.min()
        with np.errstate(invalid="ignore", divide="ignore"):
            G = np.where(k0 > 0, m * (d / (R * R)) / k0, 0.0)
        return (k0 - 1.0) * m, G
    if kind == 3:      # half-space, signed distance to the plane along the normal
        nrm = np.asarray(p, dtype=np.float64)[:, None]
        return (d * nrm).sum(0), np.broadcast_to(nrm, d.shape).copy()
    raise ValueError(kind)


def analytic_fields(scene, xyz):
    """(f, G [3, N], a) for an analytic scene (geraf_inputs.Scene)."""
    x = np.asarray(xyz, dtype=np.float64)
    best_f = np.full(x.shape[1], np.inf)
    best_G = np.zeros_like(x)
    best_a = np.zeros(x.shape[1])
    for pr in scene.prims:
        f, G = _prim_sdf(pr.kind, pr.c, pr.p, x)
        take = f < best_f
        best_f = np.where(take, f, best_f)
        best_G = np.where(take, G, best_G)
        best_a = np.where(take, pr.a, best_a)
    return best_f, best_G, best_a


# --------------------------------------------------------------------------
# Neural fields (section 5.2 "Opaque density representation" / "Signal
# representation"; App. C "Training Setup"): sinusoidal positional encoding
# (section 9.3) gamma(x) = [sin(2^k pi x), cos(2^k pi x)]_{k < L} of the
# position normalised to the cube, softplus MLP, head [f, a_logit],
# a = sigmoid(a_logit). The normal direction is grad f (section 5.2), obtained
# with three forward-mode tangents d/dx, d/dy, d/dz.
# --------------------------------------------------------------------------

def _softplus(h, beta):
    return np.maximum(h, 0.0) + np.log1p(np.exp(-beta * np.abs(h))) / beta


def _sigmoid(x):
    return 0.5 * (1.0 + np.tanh(0.5 * x))


def positional_encoding(spec, xyz):
    """gamma [6L, N] and its x-derivatives dgamma [3, 6L, N]. Feature 6k+d is
    sin(2^k pi xt_d), 6k+3+d is cos(2^k pi xt_d), xt = (x - center)/half."""
    # center and half are FP32 fields of the network description, like every
    # other input: promote their FP32 values (at octave 2^9 the FP32 rounding
    # of 0.15 m alone shifts the phase by ~2e-4 rad)
    x = np.asarray(xyz, dtype=np.float64)
    c = np.asarray(spec.center, dtype=np.float32).astype(np.float64)[:, None]
    half = np.float64(np.float32(spec.half))
    xt = (x - c) / half
    L, N = spec.n_levels, x.shape[1]
    g = np.zeros((6 * L, N))
    dg = np.zeros((3, 6 * L, N))
    for k in range(L):
        w = (2.0 ** k) * np.pi
        for d in range(3):
            g[6 * k + d] = np.sin(w * xt[d])
            g[6 * k + 3 + d] = np.cos(w * xt[d])
            dg[d, 6 * k + d] = w / half * np.cos(w * xt[d])
            dg[d, 6 * k + 3 + d] = -w / half * np.sin(w * xt[d])
    return g, dg


def bf16_round(x):
    """Round to bfloat16 (through FP32, round to nearest even), returned as FP64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + np.uint64(0x7FFF) + ((u >> np.uint64(16)) & np.uint64(1))) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def mlp_forward(spec, params, xyz, precision="fp32"):
    """Returns (f [N], G [3, N], a [N], cache). precision "bf16" is the BF16
    network: hidden-layer weights and every hidden layer's inputs (encoding,
    activations, tangents) rounded to bfloat16, sums exact (FP64); biases and
    the head weights FP32, the head reads the last BF16 activations."""
    from geraf_inputs import unpack_params
    layers = [(W.astype(np.float64), b.astype(np.float64))
              for W, b in unpack_params(spec, np.asarray(params, dtype=np.float32))]
    bf = precision == "bf16"
    r = bf16_round if bf else (lambda v: v)
    z, dz = positional_encoding(spec, xyz)
    cache = {"z": [z], "dz": [dz], "h": [], "dh": [], "precision": precision}
    for W, b in layers[:-1]:
        Wr, zr, dzr = r(W), r(z), r(dz)
        h = Wr @ zr + b[:, None]
        dh = Wr @ dzr                                  # [3, out, N]: W times each tangent
        s = _sigmoid(spec.beta * h)
        z = _softplus(h, spec.beta)
        dz = s[None] * dh
        cache["h"].append(h); cache["dh"].append(dh)
        cache["z"].append(z); cache["dz"].append(dz)
    Wh, bh = layers[-1]
    zr, dzr = r(z), r(dz)
    f = Wh[0] @ zr + bh[0]
    G = Wh[0] @ dzr                                    # [3, N]
    a = None
    if Wh.shape[0] == 2:                               # head [f, a_logit]
        a = _sigmoid(Wh[1] @ zr + bh[1])
    cache["a"] = a
    return f, G, a, cache


def mlp_backward(spec, params, cache, d_f, d_G, d_a):
    """Hand-written adjoint of mlp_forward (value + three tangents). Returns the
    gradient with respect to the packed parameters, FP64, same layout.
    For the BF16 network it is the straight-through adjoint: each rounding is
    passed through as the identity, so the products use the rounded operands
    the forward multiplied (rounded hidden weights, rounded layer inputs)."""
    from geraf_inputs import unpack_params
    layers = [(W.astype(np.float64), b.astype(np.float64))
              for W, b in unpack_params(spec, np.asarray(params, dtype=np.float32))]
    r = bf16_round if cache.get("precision") == "bf16" else (lambda v: v)
    d_f = np.asarray(d_f, np.float64)
    d_G = np.asarray(d_G, np.float64)
    grads = [None] * len(layers)
    Wh, _ = layers[-1]
    zL, dzL = r(cache["z"][-1]), r(cache["dz"][-1])
    gW = np.zeros_like(Wh)
    gW[0] = zL @ d_f + sum(dzL[d] @ d_G[d] for d in range(3))
    zbar = np.outer(Wh[0], d_f)
    if Wh.shape[0] == 2:                               # head [f, a_logit]
        a = cache["a"]
        d_logit = np.asarray(d_a, np.float64) * a * (1.0 - a)
        gW[1] = zL @ d_logit
        grads[-1] = (gW, np.array([d_f.sum(), d_logit.sum()]))
        zbar = zbar + np.outer(Wh[1], d_logit)
    else:
        grads[-1] = (gW, np.array([d_f.sum()]))
    dzbar = Wh[0][None, :, None] * d_G[:, None, :]     # [3, width, N]
    for l in range(len(layers) - 2, -1, -1):
        W = r(layers[l][0])
        h, dh = cache["h"][l], cache["dh"][l]
        s = _sigmoid(spec.beta * h)
        ds = spec.beta * s * (1.0 - s)
        dhbar = s[None] * dzbar                        # through dz = s * dh
        hbar = zbar * s + (dzbar * dh).sum(0) * ds     # through z = softplus(h) and s(h)
        zin, dzin = r(cache["z"][l]), r(cache["dz"][l])
        gW = hbar @ zin.T + sum(dhbar[d] @ dzin[d].T for d in range(3))
        grads[l] = (gW, hbar.sum(1))
        zbar = W.T @ hbar
        dzbar = W.T @ dhbar                            # [3, in, N]
    return np.concatenate([np.concatenate([gW.reshape(-1), gb]) for gW, gb in grads])


def nets_forward(nets, params, xyz, precision="fp32"):
    """The paper's two field networks (App. C, "Training Setup"; section 5.2
    "Signal representation": a separate network of the position gives the
    reflection coefficient): f and G = grad f from the SDF network, a =
    sigmoid of the reflectivity network's output, both on the same encoding of
    x. precision "bf16" applies the BF16 network reading of mlp_forward to both
    networks. Returns (f, G, a, cache)."""
    params = np.asarray(params, np.float32)
    ns = nets.sdf.n_params
    f, G, _, cs = mlp_forward(nets.sdf, params[:ns], xyz, precision=precision)
    logit, _, _, cr = mlp_forward(nets.refl, params[ns:], xyz, precision=precision)
    a = _sigmoid(logit)
    return f, G, a, {"sdf": cs, "refl": cr, "a": a}


def nets_backward(nets, params, cache, d_f, d_G, d_a):
    """Adjoint of nets_forward: gradient of the packed [SDF | reflectivity]
    parameters (FP64)."""
    params = np.asarray(params, np.float32)
    ns = nets.sdf.n_params
    gs = mlp_backward(nets.sdf, params[:ns], cache["sdf"], d_f, d_G, None)
    a = cache["a"]
    d_logit = np.asarray(d_a, np.float64) * a * (1.0 - a)
    n = a.shape[0]
    gr = mlp_backward(nets.refl, params[ns:], cache["refl"], d_logit, np.zeros((3, n)), None)
    return np.concatenate([gs, gr])


# --------------------------------------------------------------------------
# Lensless alpha blending (section 5.2 "Discretization"; section 6 "Lensless
# Alpha Blending"; App. B).
#   Phi_s(x) = 1 / (1 + exp(-s x))  (logistic CDF, NeuS S-density)
#   alpha_k = max((Phi_s(f_k) - Phi_s(f_{k+1})) / Phi_s(f_k), 0)  along a primary
#             column (NeuS discretisation of 1 - exp(-int rho du)); last depth 0
#   T_k = prod_{m<k} (1 - alpha_m)
#   w_k = a_k alpha_k A'_tx               (antenna-independent part of Eq. signal_amp_tracing)
#   t_eff_k = T_k + Phi_s(f(x_apr))       (primary origin term of the T correction)
#   c_ant_i = Phi_s(f(a_i))               (real origin term; both stop-gradient)
# The ratio Phi_{k+1}/Phi_k is formed as exp(log Phi_{k+1} - log Phi_k).
# --------------------------------------------------------------------------

def _log_cdf(x):
    return -np.logaddexp(0.0, -x)


def cdf(s, f):
    return np.exp(_log_cdf(s * np.asarray(f, np.float64)))


def blend(sdf, refl, n_ray, n_z, sdf_apr, sdf_ant, s, a_tx, keep=None):
    """keep (optional, per sample) multiplies w: a sample with keep = 0 still
    ends the interval of the sample before it and its own alpha still
    attenuates T, but it reflects nothing."""
    f = np.asarray(sdf, np.float64).reshape(n_z, n_ray)
    a = np.asarray(refl, np.float64).reshape(n_z, n_ray)
    if keep is not None:
        a = a * np.asarray(keep, np.float64).reshape(n_z, n_ray)
    lc = _log_cdf(s * f)
    alpha = np.zeros((n_z, n_ray))
    alpha[:-1] = np.maximum(-np.expm1(lc[1:] - lc[:-1]), 0.0)
    T = np.ones((n_z, n_ray))
    for k in range(1, n_z):
        T[k] = T[k - 1] * (1.0 - alpha[k - 1])
    w = a * alpha * a_tx
    t_eff = T + cdf(s, sdf_apr)[None, :]
    c_ant = cdf(s, sdf_ant)
    return (alpha.reshape(-1), T.reshape(-1), w.reshape(-1), t_eff.reshape(-1), c_ant)


def blend_backward(sdf, refl, n_ray, n_z, s, a_tx, d_w, d_teff, keep=None):
    """Adjoint of blend for (w, t_eff); origin terms carry no gradient
    (section 6, stop-gradient on the ray-origin sigmoid-SDF).
    Returns (d_sdf [N], d_refl [N], d_s, d_a_tx)."""
    f = np.asarray(sdf, np.float64).reshape(n_z, n_ray)
    a = np.asarray(refl, np.float64).reshape(n_z, n_ray)
    alpha, T, _, _, _ = blend(sdf, refl, n_ray, n_z, np.zeros(n_ray), np.zeros(1), s, a_tx)
    alpha = alpha.reshape(n_z, n_ray); T = T.reshape(n_z, n_ray)
    dw = np.asarray(d_w, np.float64).reshape(n_z, n_ray)
    if keep is not None:                              # w = keep a alpha A'_tx
        dw = dw * np.asarray(keep, np.float64).reshape(n_z, n_ray)
    dt = np.asarray(d_teff, np.float64).reshape(n_z, n_ray)
    d_alpha = dw * a * a_tx
    d_a = dw * alpha * a_tx
    d_atx = float((dw * a * alpha).sum())
    # reverse scan of T_{k+1} = T_k (1 - alpha_k)
    gT_next = np.zeros(n_ray)
    for k in range(n_z - 1, -1, -1):
        if k < n_z - 1:
            d_alpha[k] -= gT_next * T[k]
            gT = dt[k] + gT_next * (1.0 - alpha[k])
        else:
            gT = dt[k]
        gT_next = gT
    # alpha_k = 1 - R, R = Phi_{k+1}/Phi_k, active where f_{k+1} < f_k
    d_f = np.zeros((n_z, n_ray))
    x0, x1 = s * f[:-1], s * f[1:]
    R = np.exp(_log_cdf(x1) - _log_cdf(x0))
    act = f[1:] < f[:-1]
    sig0, sig1 = np.exp(_log_cdf(-x0)), np.exp(_log_cdf(-x1))   # 1 - Phi
    g = np.where(act, d_alpha[:-1], 0.0)
    d_f[:-1] += g * R * s * sig0
    d_f[1:] -= g * R * s * sig1
    d_s = float((-g * R * (f[1:] * sig1 - f[:-1] * sig0)).sum())
    return d_f.reshape(-1), d_a.reshape(-1), d_s, d_atx


# --------------------------------------------------------------------------
# Phasor sums (C, FP64): signal tracing and matched filter with adjoints.
# --------------------------------------------------------------------------
_lib = None


def _clib():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(_build.build())
        P = ctypes.POINTER(ctypes.c_double)
        L, I, D = ctypes.c_long, ctypes.c_int, ctypes.c_double
        lib.oracle_render.argtypes = [L, P, P, P, P, P, P, P, P, L, P, P, P, P, D, D, L, I, P, P]
        lib.oracle_render_backward.argtypes = [L, P, P, P, P, P, P, P, P, L, P, P, P, P, D, D, L, I,
                                               P, P, P, P, P, P, P]
        lib.oracle_filter.argtypes = [L, P, P, P, L, P, P, P, D, D, L, P, P, P, P, P]
        lib.oracle_filter_backward.argtypes = [L, P, P, P, L, P, P, P, D, D, L, P, P, P, P, P]
        _lib = lib
    return _lib


def _d(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return a


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def render(xyz, G, w, t_eff, ant, c_ant, band, use_dir=True):
    """Signal tracing s [N_ant, N_f] complex128 (section 5.1, Eq. ref_sim)."""
    x, g = _d(xyz), _d(G)
    w, t, A, c = _d(w), _d(t_eff), _d(ant), _d(c_ant)
    n_pts, n_ant, n_f = x.shape[1], A.shape[1], band.n_f
    sr = np.zeros((n_ant, n_f)); si = np.zeros((n_ant, n_f))
    keep = [x, g, w, t, A, c]
    _clib().oracle_render(n_pts, _p(x[0]), _p(x[1]), _p(x[2]), _p(g[0]), _p(g[1]), _p(g[2]),
                          _p(w), _p(t), n_ant, _p(A[0]), _p(A[1]), _p(A[2]), _p(c),
                          band.f0, band.df, n_f, int(bool(use_dir)), _p(sr), _p(si))
    del keep
    return sr + 1j * si


def render_backward(xyz, G, w, t_eff, ant, c_ant, band, g_s, use_dir=True):
    """Adjoint of render for g_s = dL/dRe s + j dL/dIm s.
    Returns (d_w [N], d_teff [N], d_G [3, N])."""
    x, g = _d(xyz), _d(G)
    w, t, A, c = _d(w), _d(t_eff), _d(ant), _d(c_ant)
    gs = np.asarray(g_s)
    gr, gi = _d(gs.real), _d(gs.imag)
    n_pts, n_ant, n_f = x.shape[1], A.shape[1], band.n_f
    dw, dt = np.zeros(n_pts), np.zeros(n_pts)
    dG = np.zeros((3, n_pts))
    _clib().oracle_render_backward(n_pts, _p(x[0]), _p(x[1]), _p(x[2]), _p(g[0]), _p(g[1]), _p(g[2]),
                                   _p(w), _p(t), n_ant, _p(A[0]), _p(A[1]), _p(A[2]), _p(c),
                                   band.f0, band.df, n_f, int(bool(use_dir)), _p(gr), _p(gi),
                                   _p(dw), _p(dt), _p(dG[0]), _p(dG[1]), _p(dG[2]))
    return dw, dt, dG


def filter_forward(s, ant, vox, band):
    """Matched filter: (M [N_vox] complex128, P [N_vox]) (section 3, Eq. mf-sm)."""
    s = np.asarray(s)
    sr, si = _d(s.real), _d(s.imag)
    A, V = _d(ant), _d(vox)
    n_vox, n_ant = V.shape[1], A.shape[1]
    Mr, Mi, P = np.zeros(n_vox), np.zeros(n_vox), np.zeros(n_vox)
    _clib().oracle_filter(n_vox, _p(V[0]), _p(V[1]), _p(V[2]), n_ant, _p(A[0]), _p(A[1]), _p(A[2]),
                          band.f0, band.df, band.n_f, _p(sr), _p(si), _p(Mr), _p(Mi), _p(P))
    return Mr + 1j * Mi, P


def filter_backward(M, dP, ant, vox, band):
    """Adjoint of |matched filter|: g [N_ant, N_f] complex128 (App. A.5)."""
    M = np.asarray(M)
    Mr, Mi, d = _d(M.real), _d(M.imag), _d(dP)
    A, V = _d(ant), _d(vox)
    n_vox, n_ant = V.shape[1], A.shape[1]
    gr, gi = np.zeros((n_ant, band.n_f)), np.zeros((n_ant, band.n_f))
    _clib().oracle_filter_backward(n_vox, _p(V[0]), _p(V[1]), _p(V[2]), n_ant, _p(A[0]), _p(A[1]),
                                   _p(A[2]), band.f0, band.df, band.n_f, _p(Mr), _p(Mi), _p(d),
                                   _p(gr), _p(gi))
    return gr + 1j * gi


def dynamic_mask(P, history, p_ref, rho_hi, rho_lo):
    """Dynamic loss masking (section 6 "Dynamic loss masking"): a voxel whose
    matched-filter response was high in an earlier iteration (history = the
    running maximum of its earlier P >= rho_hi * p_ref) but is low now
    (P < rho_lo * p_ref) is left out of the loss. Returns (mask [N] in {0, 1},
    the updated history max(history, P)). The thresholds are relative to p_ref,
    the maximum of the target heatmap (the paper gives no values)."""
    P = np.asarray(P, np.float64)
    H = np.asarray(history, np.float64)
    drop = (H >= rho_hi * p_ref) & (P < rho_lo * p_ref)
    return np.where(drop, 0.0, 1.0), np.maximum(H, P)


def heatmap_loss(P, target, mask=None):
    """L2 heatmap loss (section 4, step 5): L = sum_v m_v (P_v - P*_v)^2 and dL/dP."""
    P = np.asarray(P, np.float64)
    t = np.asarray(target, np.float64)
    m = np.ones_like(P) if mask is None else np.asarray(mask, np.float64)
    r = P - t
    return float((m * r * r).sum()), 2.0 * m * r


# --------------------------------------------------------------------------
# Learned proposal sampler (the paper is silent; its definition here follows
# the proposal-network idea of mip-NeRF 360: a small network predicts, per
# primary column, a depth distribution from which the lensless samples are
# drawn; it is trained online on the blended weights of the method itself).
#   grid cell (gx, gy, gz) of a G0 x G1 x G2 grid over the sample cube holds an
#   F-dim feature (FP16 values); an MLP (n_hidden layers of `width`,
#   softplus(beta) like the field network, output 1 logit) maps it to a logit;
#   per grid column q_k = (1 - eps) softmax(logits)_k + eps / G2.
#   Sampling column (ix, iy) of the fine grid uses grid column
#   (ix * G0 // nx, iy * G1 // ny). Integer CDF: c_k = max(1, floor(q_k 2^20)),
#   C_{k+1} = C_k + c_k, W = C_G2; sample j of D: m_j = SplitMix64 output
#   (step<<42 | 3<<40 | ray*D + j) >> 40 (24 bits), u_j = ((j<<24) + m_j) W //
#   (D<<24); k = the cell with C_k <= u_j < C_{k+1}; depth
#   z = z0 + (k + (u_j - C_k + 0.5)/c_k) * pz_cell in FP64, rounded to FP32.
# --------------------------------------------------------------------------

def proposal_shapes(feat, width, n_hidden):
    dims = [feat] + [width] * n_hidden
    return [(dims[l + 1], dims[l]) for l in range(n_hidden)] + [(1, width)]


def _unpack(shapes, params):
    out, off = [], 0
    params = np.asarray(params, dtype=np.float32).astype(np.float64)
    for o, i in shapes:
        W = params[off:off + o * i].reshape(o, i); off += o * i
        b = params[off:off + o]; off += o
        out.append((W, b))
    return out


def proposal_logits(features, params, width, n_hidden, beta):
    """features [n_cells, F] (FP16 values) -> logits [n_cells] and a cache."""
    Fe = np.asarray(features, dtype=np.float16).astype(np.float64)
    layers = _unpack(proposal_shapes(Fe.shape[1], width, n_hidden), params)
    z = Fe.T
    cache = {"z": [z], "h": []}
    for W, b in layers[:-1]:
        h = W @ z + b[:, None]
        z = _softplus(h, beta)
        cache["h"].append(h); cache["z"].append(z)
    W, b = layers[-1]
    return (W @ z + b[:, None])[0], cache


def proposal_q(logits, gshape, eps):
    """Per grid column depth distribution q [G2, G1, G0] from logits laid out
    [G2][G1][G0] (cell index (gz*G1 + gy)*G0 + gx)."""
    G0, G1, G2 = gshape
    L = np.asarray(logits, np.float64).reshape(G2, G1, G0)
    e = np.exp(L - L.max(0, keepdims=True))
    sm = e / e.sum(0, keepdims=True)
    return (1.0 - eps) * sm + eps / G2


def proposal_sample(grid, gshape, q_f32, D, seed, step):
    """Inverse-CDF depth samples per fine column from FP32 probabilities
    q_f32 [G2, G1, G0]. Returns (xyz [3, n_ray*D] float32, apr, cell idx int32)."""
    nx, ny, _ = grid.n
    G0, G1, G2 = gshape
    n_ray = nx * ny
    ray = np.arange(n_ray, dtype=np.int64)
    ix, iy = ray % nx, ray // nx
    ux = uniform01(seed, step, 0, ray)
    uy = uniform01(seed, step, 1, ray)
    xr = _coord(grid.lo[0], ix, ux, grid.pitch[0])
    yr = _coord(grid.lo[1], iy, uy, grid.pitch[1])
    gxi, gyi = ix * G0 // nx, iy * G1 // ny
    q = np.asarray(q_f32, dtype=np.float32)
    c = np.maximum(np.floor(q.astype(np.float64) * 2.0 ** 20), 1.0).astype(np.int64)   # [G2, G1, G0]
    C = np.concatenate([np.zeros((1, G1, G0), np.int64), np.cumsum(c, 0)], 0)         # [G2+1, G1, G0]
    Cr = C[:, gyi, gxi]                                                                  # [G2+1, n_ray]
    cr = c[:, gyi, gxi]
    W = Cr[-1]
    j = np.arange(D, dtype=np.int64)
    idx = (ray[:, None] * D + j[None, :]).astype(np.uint64)
    k = (np.uint64(step) << np.uint64(42)) | (np.uint64(3) << np.uint64(40)) | idx
    m = (splitmix64(seed, k) >> np.uint64(40)).astype(np.int64)
    u = ((j[None, :] << 24) + m) * W[:, None] // (np.int64(D) << 24)                   # [n_ray, D]
    cell = np.empty((n_ray, D), np.int64)
    for r in range(n_ray):
        cell[r] = np.searchsorted(Cr[:, r], u[r], side="right") - 1
    Ck = np.take_along_axis(Cr.T, cell, 1)
    ck = np.take_along_axis(cr.T, cell, 1)
    frac = (u - Ck).astype(np.float64) + 0.5
    frac = frac / ck.astype(np.float64)
    pz_cell = np.float64(np.float32(grid.pitch[2] * grid.n[2] / G2))
    zc = np.float64(np.float32(grid.lo[2])) + (cell.astype(np.float64) + frac) * pz_cell
    xyz = np.empty((3, D * n_ray), np.float32)        # depth-major: point = j * n_ray + ray
    xyz[0] = np.tile(xr, D)
    xyz[1] = np.tile(yr, D)
    xyz[2] = zc.T.reshape(-1).astype(np.float32)
    apr = np.stack([xr, yr, np.full(n_ray, np.float32(grid.aperture_z))]).astype(np.float32)
    gcell = (cell * G1 + gyi[:, None]) * G0 + gxi[:, None]
    return xyz, apr, gcell.T.reshape(-1).astype(np.int32)


def sample_cells(grid, gshape, q_f32, m, r_max, seed, step, dilate=0):
    """Samples of the m cells of largest q per grid column (the learned
    sampler's cell selection): the STRATIFIED grid's own points of the kept
    cells (taken from `sample`, so bit-exact with the dense grid), in depth
    order; after each of the first r_max runs of consecutive kept cells (not
    after the last cell) the first fine depth of the next cell closes the run;
    the column is padded to n_out = m s + r_max with its last sample. Cells are
    ranked by the largest q within `dilate` cells, then their own q, then the
    lower index. keep = 1
    on kept-cell samples, 0 on the others; idx = the grid cell of each sample.
    Returns (xyz [3, n_ray n_out], apr [3, n_ray], idx, keep, n_out)."""
    G0, G1, G2 = gshape
    nx, ny, nz = grid.n
    s_fine = nz // G2
    n_out = m * s_fine + r_max
    n_ray = nx * ny
    dense, apr = sample(grid, 1, seed, step)          # STRATIFIED, [3, nz n_ray]
    q = np.asarray(q_f32, np.float32).reshape(G2, G1 * G0)
    tables = []
    for col in range(G1 * G0):
        qc = q[:, col].astype(np.float64)
        qd = np.array([qc[max(0, k - dilate):k + dilate + 1].max() for k in range(G2)])
        order = np.lexsort((np.arange(G2), -qc, -qd))    # dilated q, own q, lower cell
        cells = sorted(int(c) for c in order[:m])
        t, runs = [], 0
        for i, c in enumerate(cells):
            t += [(c * s_fine + d, 1) for d in range(s_fine)]
            run_end = i + 1 == m or cells[i + 1] != c + 1
            if run_end and runs < r_max and c + 1 < G2:
                t.append(((c + 1) * s_fine, 0))
                runs += 1
        while len(t) < n_out:
            t.append((t[-1][0], 0))
        tables.append(t)
    n = n_ray * n_out
    xyz = np.zeros((3, n), np.float32)
    idx = np.zeros(n, np.int32)
    keep = np.zeros(n, np.float32)
    for ray in range(n_ray):
        ix, iy = ray % nx, ray // nx
        col = (iy * G1 // ny) * G0 + (ix * G0 // nx)
        for slot, (kz, kp) in enumerate(tables[col]):
            p = slot * n_ray + ray
            xyz[:, p] = dense[:, kz * n_ray + ray]
            idx[p] = (kz // s_fine) * (G0 * G1) + col
            keep[p] = kp
    return xyz, apr, idx, keep, n_out


def proposal_targets(omega, idx, n_cells):
    """Histogram of the blended geometric weights omega = T alpha over grid cells."""
    return np.bincount(np.asarray(idx, np.int64), weights=np.asarray(omega, np.float64), minlength=n_cells)


def proposal_loss(logits, gshape, eps, hist):
    """Sum over grid columns of KL(p || q), p = normalised weight histogram of
    the column (columns without weight are skipped); returns (loss, dL/dlogits)."""
    G0, G1, G2 = gshape
    L = np.asarray(logits, np.float64).reshape(G2, G1, G0)
    e = np.exp(L - L.max(0, keepdims=True))
    sm = e / e.sum(0, keepdims=True)
    q = (1.0 - eps) * sm + eps / G2
    h = np.asarray(hist, np.float64).reshape(G2, G1, G0)
    tot = h.sum(0, keepdims=True)
    has = tot > 0
    p = np.where(has, h / np.where(has, tot, 1.0), 0.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        kl = np.where(p > 0, p * (np.log(p) - np.log(q)), 0.0).sum()
    r = p / q
    dz = (1.0 - eps) * sm * (-r + (r * sm).sum(0, keepdims=True))
    dz = np.where(has, dz, 0.0)
    return float(kl), dz.reshape(-1)


def proposal_backward(features, params, width, n_hidden, beta, cache, d_logits):
    """Adjoint of proposal_logits: (d_params FP64 packed, d_features [n_cells, F])."""
    Fe = np.asarray(features, dtype=np.float16).astype(np.float64)
    layers = _unpack(proposal_shapes(Fe.shape[1], width, n_hidden), params)
    g = np.asarray(d_logits, np.float64)[None, :]
    W, b = layers[-1]
    grads = [None] * len(layers)
    grads[-1] = (g @ cache["z"][-1].T, g.sum(1))
    zbar = W.T @ g
    for l in range(len(layers) - 2, -1, -1):
        W, b = layers[l]
        h = cache["h"][l]
        hbar = zbar * _sigmoid(beta * h)
        grads[l] = (hbar @ cache["z"][l].T, hbar.sum(1))
        zbar = W.T @ hbar
    d_params = np.concatenate([np.concatenate([gW.reshape(-1), gb]) for gW, gb in grads])
    return d_params, zbar.T
