"""CUDA path vs the FP64 oracle, stage by stage, through the C ABI.

Each stage gets identical FP32 inputs on both sides (the oracle promotes them
to FP64). Tolerances: integer/bit work is exact; FP32 outputs must match to
relative L2 <= 1e-5 (the FP32-path bound), a few gradient outputs whose
directional-factor branch can flip within FP32 rounding of 2c^2 - 1 get 3e-5.
Sizes are ragged on purpose: points not a multiple of the point tile, antennas
not a multiple of the CTA's antenna slice, bins not a multiple of 32.
"""
import numpy as np
import pytest
import torch

import geraf_inputs as gi
from brick_order import brick_order
from parity_helpers import away_from_clamp_kink, away_from_directional_kink

pytestmark = pytest.mark.gpu

TOL = 1e-5


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.complex128 if np.iscomplexobj(a) else np.float64)
    b = np.asarray(b, dtype=a.dtype)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2605_29097_gb300 import _build
    _build.build()
    import paper_2605_29097_gb300 as G
    return G


def cu(x):
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float32), device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def _band(G, b, method=0):
    return G.Band(b.f0, b.df, b.n_f, method)


# both ways of stepping across the bins, forced (the default picks by n_f)
METHODS = [pytest.param(1, id="recurrence"), pytest.param(2, id="chebyshev")]


def _scene_points(rng, n, centre=(0.0, 0.0, 0.15), half=0.05):
    xyz = (np.array(centre)[:, None] + rng.uniform(-half, half, (3, n))).astype(np.float32)
    grad = rng.standard_normal((3, n)).astype(np.float32)
    grad[:, ::17] = 0.0                              # some isotropic points
    w = rng.uniform(0.0, 1.0, n).astype(np.float32)
    t_eff = rng.uniform(0.3, 2.0, n).astype(np.float32)
    return xyz, grad, w, t_eff


# ----------------------------------------------------------------- sampling
@pytest.mark.parametrize("mode", [gi.SAMPLE_UNIFORM, gi.SAMPLE_STRATIFIED])
def test_sample_bit_exact(G, oracle, mode):
    g = gi.cube_grid((0.0, 0.0, 0.15), 0.1, (33, 17, 29))
    grid = G.make_grid(g.lo, g.pitch, g.n, g.aperture_z)
    xyz, apr = G.geraf_sample(grid, mode, seed=1234, step=7)
    oxyz, oapr = oracle.sample(g, mode, seed=1234, step=7)
    np.testing.assert_array_equal(host(xyz).view(np.uint32), oxyz.view(np.uint32))
    np.testing.assert_array_equal(host(apr).view(np.uint32), oapr.view(np.uint32))


def test_sample_bit_exact_full_size_spots(G, oracle):
    """128^3 stratified (the MLP workload's sampling): every point from the
    CUDA path equals the oracle at 20 000 random indices."""
    g = gi.cube_grid((0.0, 0.0, 0.15), 0.1, (128, 128, 128))
    grid = G.make_grid(g.lo, g.pitch, g.n)
    xyz, _ = G.geraf_sample(grid, gi.SAMPLE_STRATIFIED, seed=3, step=2)
    full, _ = oracle.sample(g, gi.SAMPLE_STRATIFIED, seed=3, step=2)
    idx = np.random.default_rng(0).integers(0, g.n_pts, 20000)
    np.testing.assert_array_equal(host(xyz)[:, idx].view(np.uint32), full[:, idx].view(np.uint32))


# ----------------------------------------------------------- analytic fields
def test_analytic_fields(G, oracle):
    rng = np.random.default_rng(1)
    sc = gi.Scene([gi.Prim(gi.PRIM_SPHERE, 0.9, (0.0, 0.0, 0.15), (0.03, 0, 0)),
                   gi.Prim(gi.PRIM_BOX, 0.5, (0.02, 0.01, 0.13), (0.01, 0.015, 0.008)),
                   gi.Prim(gi.PRIM_ELLIPSOID, 0.3, (-0.02, 0.0, 0.17), (0.02, 0.01, 0.015)),
                   gi.Prim(gi.PRIM_HALFSPACE, 0.7, (0.0, 0.0, 0.195), (0.0, 0.0, -1.0))])
    xyz = (np.array([0, 0, 0.15])[:, None] + rng.uniform(-0.05, 0.05, (3, 5001))).astype(np.float32)
    f, g, a, _ = G.geraf_fields(G.AnalyticField(cu(sc.packed())), cu(xyz))
    of, og, oa = oracle.analytic_fields(sc, xyz)
    np.testing.assert_allclose(host(f), of, rtol=0, atol=2e-8)
    assert np.mean(np.abs(host(g) - og).max(0) < 1e-5) > 0.999
    np.testing.assert_array_equal(host(a), oa.astype(np.float32))


# -------------------------------------------------------------------- blend
def test_blend_and_backward(G, oracle):
    rng = np.random.default_rng(2)
    n_ray, n_z, n_ant = 301, 37, 19
    z = np.linspace(0.1, 0.2, n_z)
    sdf = (0.15 - z[:, None] + 0.01 * rng.standard_normal((n_z, n_ray))).astype(np.float32).reshape(-1)
    refl = rng.uniform(0.2, 1.0, n_ray * n_z).astype(np.float32)
    sdf_apr = rng.uniform(0.0, 0.02, n_ray).astype(np.float32)
    sdf_ant = rng.uniform(-0.005, 0.02, n_ant).astype(np.float32)
    s, atx = 300.0, 1.3
    out = G.geraf_blend(cu(sdf), cu(refl), n_ray, n_z, cu(sdf_apr), cu(sdf_ant), s, atx)
    ref = oracle.blend(sdf, refl, n_ray, n_z, sdf_apr, sdf_ant, np.float32(s), np.float32(atx))
    for name, got, want in zip(["alpha", "T", "w", "t_eff", "c_ant"], out, ref):
        assert rel_l2(host(got), want) < TOL, name
    d_w = rng.standard_normal(n_ray * n_z).astype(np.float32)
    d_t = rng.standard_normal(n_ray * n_z).astype(np.float32)
    d_sdf, d_refl, d_sc = G.geraf_blend_backward(cu(sdf), cu(refl), out[0], out[1], n_ray, n_z, s, atx,
                                                 cu(d_w), cu(d_t))
    od_f, od_a, od_s, od_atx = oracle.blend_backward(sdf, refl, n_ray, n_z, np.float32(s), np.float32(atx), d_w, d_t)
    assert rel_l2(host(d_sdf), od_f) < 1e-4   # s * Phi(1-Phi) amplifies FP32 alpha rounding
    assert rel_l2(host(d_refl), od_a) < TOL
    np.testing.assert_allclose(host(d_sc), [od_s, od_atx], rtol=1e-4)


# ------------------------------------------------------------------- render
@pytest.mark.parametrize("n_pts,n_ant_side,n_f,directional", [
    (5003, (10, 10), 45, True),       # G = 2 with a 13-bin tail; 100 antennas
    (777, (7, 5), 32, True),          # G = 1
    (2049, (9, 9), 128, False),       # Chebyshev moments, isotropic
    (4099, (12, 11), 256, True),      # Chebyshev: 132 antennas over two 128-antenna CTAs, ragged point tile
    (1, (3, 1), 7, True),             # single point, tiny band
])
@pytest.mark.parametrize("method", METHODS)
def test_render(G, oracle, n_pts, n_ant_side, n_f, directional, method):
    rng = np.random.default_rng(n_pts)
    xyz, grad, w, t_eff = _scene_points(rng, n_pts)
    ant = gi.antenna_array(*n_ant_side, 0.002)
    c_ant = rng.uniform(0.2, 1.0, ant.shape[1]).astype(np.float32)
    b = gi.band(77e9, 81e9, n_f)
    s = G.geraf_render(cu(xyz), cu(grad), cu(w), cu(t_eff), cu(ant), cu(c_ant), _band(G, b, method), directional)
    G.geraf_poll_device_error()
    want = oracle.render(xyz, grad, w, t_eff, ant, c_ant, b, use_dir=directional)
    assert rel_l2(host(s), want) < TOL


# Range spreads that put the Chebyshev order in the 32- and 64-order kernel
# instances and above its 64-term cap (the direct recurrence kernels run above
# it; the choice is made on the device), over 4 GHz: a 0.24 m cube -> about 27
# terms, a 0.5 m cube -> about 44, a 1 m cube -> above 64.
SPREADS = [((0.0, 0.0, 0.30), 0.12), ((0.0, 0.0, 0.35), 0.25), ((0.0, 0.0, 0.60), 0.50)]


@pytest.mark.parametrize("centre,half", SPREADS)
def test_render_range_spread(G, oracle, centre, half):
    rng = np.random.default_rng(11)
    n_pts, n_f = 3000, 128
    xyz, grad, w, t_eff = _scene_points(rng, n_pts, centre, half)
    ant = gi.antenna_array(10, 9, 0.002)
    c_ant = rng.uniform(0.2, 1.0, ant.shape[1]).astype(np.float32)
    b = gi.band(77e9, 81e9, n_f)
    s = G.geraf_render(cu(xyz), cu(grad), cu(w), cu(t_eff), cu(ant), cu(c_ant), _band(G, b), True)
    G.geraf_poll_device_error()
    want = oracle.render(xyz, grad, w, t_eff, ant, c_ant, b)
    assert rel_l2(host(s), want) < TOL
    g = gi.complex_normal(rng, (ant.shape[1], n_f)).astype(np.complex64)
    d_w, d_t, d_g = G.geraf_render_backward(cu(xyz), cu(grad), cu(w), cu(t_eff), cu(ant), cu(c_ant),
                                            _band(G, b), torch.as_tensor(g, device="cuda"))
    G.geraf_poll_device_error()
    ow, ot, og = oracle.render_backward(xyz, grad, w, t_eff, ant, c_ant, b, g)
    assert rel_l2(host(d_w), ow) < TOL
    kt = away_from_clamp_kink(t_eff, c_ant)     # d_t: away from the clamp's kinks
    assert rel_l2(host(d_t)[kt], ot[kt]) < TOL
    assert rel_l2(host(d_g), og) < 3 * TOL


@pytest.mark.parametrize("centre,half", SPREADS)
def test_filter_range_spread(G, oracle, centre, half):
    rng = np.random.default_rng(12)
    n_vox, n_f = 2500, 128
    ant = gi.antenna_array(9, 10, 0.002)
    s = gi.complex_normal(rng, (ant.shape[1], n_f)).astype(np.complex64)
    vox = (np.array(centre)[:, None] + rng.uniform(-half, half, (3, n_vox))).astype(np.float32)
    b = gi.band(77e9, 81e9, n_f)
    P, M, _, _ = G.geraf_filter(torch.as_tensor(s, device="cuda"), cu(ant), _band(G, b), cu(vox))
    G.geraf_poll_device_error()
    oM, oP = oracle.filter_forward(s, ant, vox, b)
    assert rel_l2(host(M), oM) < TOL
    d_P = rng.standard_normal(n_vox).astype(np.float32)
    g = G.geraf_filter_backward(cu(ant), _band(G, b), cu(vox), M, cu(d_P))
    G.geraf_poll_device_error()
    og = oracle.filter_backward(host(M), d_P, ant, vox, b)
    assert rel_l2(host(g), og) < TOL


@pytest.mark.parametrize("n_f", [40, 70, 256])
@pytest.mark.parametrize("method", METHODS)
def test_render_backward(G, oracle, n_f, method):
    rng = np.random.default_rng(5)
    n_pts = 1203
    xyz, grad, w, t_eff = _scene_points(rng, n_pts)
    ant = gi.antenna_array(7, 9, 0.002)
    c_ant = rng.uniform(0.2, 1.0, ant.shape[1]).astype(np.float32)
    b = gi.band(77e9, 81e9, n_f)
    g = gi.complex_normal(rng, (ant.shape[1], b.n_f)).astype(np.complex64)
    d_w, d_t, d_g = G.geraf_render_backward(cu(xyz), cu(grad), cu(w), cu(t_eff), cu(ant), cu(c_ant),
                                            _band(G, b, method), torch.as_tensor(g, device="cuda"))
    G.geraf_poll_device_error()
    ow, ot, og = oracle.render_backward(xyz, grad, w, t_eff, ant, c_ant, b, g)
    assert rel_l2(host(d_w), ow) < TOL
    kt = away_from_clamp_kink(t_eff, c_ant)     # d_t: away from the clamp's kinks
    assert rel_l2(host(d_t)[kt], ot[kt]) < TOL
    assert rel_l2(host(d_g), og) < 3 * TOL


# ------------------------------------------------------------------- filter
@pytest.mark.parametrize("n_vox,n_ant_side,n_f", [(3001, (6, 7), 40), (256, (16, 16), 32), (1, (2, 2), 3),
                                                  (3001, (6, 7), 64), (2000, (12, 11), 200)])
@pytest.mark.parametrize("method", METHODS)
def test_filter_and_backward(G, oracle, n_vox, n_ant_side, n_f, method):
    rng = np.random.default_rng(n_vox)
    ant = gi.antenna_array(*n_ant_side, 0.002)
    b = gi.band(77e9, 81e9, n_f)
    s = gi.complex_normal(rng, (ant.shape[1], n_f)).astype(np.complex64)
    vox = (np.array([0, 0, 0.15])[:, None] + rng.uniform(-0.05, 0.05, (3, n_vox))).astype(np.float32)
    target = rng.uniform(0, 5, n_vox).astype(np.float32)
    P, M, loss, dP = G.geraf_filter(torch.as_tensor(s, device="cuda"), cu(ant), _band(G, b, method), cu(vox),
                                    cu(target))
    G.geraf_poll_device_error()
    oM, oP = oracle.filter_forward(s, ant, vox, b)
    assert rel_l2(host(M), oM) < TOL
    assert rel_l2(host(P), oP) < TOL
    oL, odP = oracle.heatmap_loss(oP, target)
    np.testing.assert_allclose(float(loss), oL, rtol=1e-5)
    assert rel_l2(host(dP), odP) < 1e-4
    # backward from the kernel's own M (the oracle gets the same FP32 M)
    d_P = rng.standard_normal(n_vox).astype(np.float32)
    g = G.geraf_filter_backward(cu(ant), _band(G, b, method), cu(vox), M, cu(d_P))
    G.geraf_poll_device_error()
    og = oracle.filter_backward(host(M), d_P, ant, vox, b)
    assert rel_l2(host(g), og) < TOL


def _host_order(xyz, ant, b, eps=1e-7, kmax=64):
    """Chebyshev order from the bounding box and the Bessel tail, on the host
    (scipy's J_k): the rule the device plan follows, stated independently.
    Each antenna's interval runs from its nearest to its farthest range to the
    box, about its own centre; the half range dr is the largest half span over
    the antennas, and the largest Bessel argument is pi (n_f - 1) (2 df / c) dr
    (bin offsets of at most (n_f - 1) / 2 from the band's centre)."""
    special = pytest.importorskip("scipy.special")
    lo, hi = xyz.min(1).astype(np.float64), xyz.max(1).astype(np.float64)
    a = ant.astype(np.float64)
    near = np.sqrt((np.maximum(np.maximum(lo[:, None] - a, a - hi[:, None]), 0.0) ** 2).sum(0))
    far = np.sqrt((np.maximum(np.abs(a - lo[:, None]), np.abs(hi[:, None] - a)) ** 2).sum(0))
    dr = max((0.5 * (far - near)).max() * 1.001 + 1e-6, 1e-5)
    amax = np.pi * (b.n_f - 1) * (2 * b.df / 299792458.0) * dr
    J = np.abs(special.jv(np.arange(kmax + 8), amax))
    tail = np.cumsum((2 * J)[::-1])[::-1]            # tail[k] = sum_{m >= k} 2 |J_m|
    above = np.nonzero(tail > eps)[0]
    K = max(int(above[-1]) + 1, 2)
    return 0 if K > kmax else K


@pytest.mark.parametrize("centre,half", SPREADS)
def test_chebyshev_order(G, centre, half):
    rng = np.random.default_rng(13)
    xyz = (np.array(centre)[:, None] + rng.uniform(-half, half, (3, 4000))).astype(np.float32)
    ant = gi.antenna_array(16, 16, 0.002)
    b = gi.band(77e9, 81e9, 128)
    want = _host_order(xyz, ant, b)
    got = G.geraf_chebyshev_order(cu(xyz), cu(ant), _band(G, b))
    assert abs(got - want) <= 1 and (got == 0) == (want == 0), (got, want)
    b32 = gi.band(77e9, 81e9, 32)
    if want:
        assert 20 <= got <= 64
        # the order follows the band's span, not its bin count
        assert G.geraf_chebyshev_order(cu(xyz), cu(ant), _band(G, b32, 2)) == got
    else:
        assert got == 0                               # above the cap: the recurrence runs
    assert G.geraf_chebyshev_order(cu(xyz), cu(ant), _band(G, b, 1)) == 0
    assert G.geraf_chebyshev_order(cu(xyz), cu(ant), _band(G, b32)) == 0      # auto: recurrence below 64 bins


# ------------------------------------------- the analytic-scene workload chain
def test_sphere_and_point_reflector_chain(G, oracle):
    """32^3 uniform samples of a 10 cm cube, sphere r = 3 cm at 15 cm plus a
    point reflector, 16x16 array at 2 mm, 32 bins over 77-81 GHz: every stage on
    the GPU from the GPU's own previous stage, compared with the oracle run on
    the same FP32 stage inputs, and the final heatmap against the all-oracle
    chain."""
    wl = gi.workload("c1")
    g = wl.grid
    grid = G.make_grid(g.lo, g.pitch, g.n, g.aperture_z)
    xyz, apr = G.geraf_sample(grid, gi.SAMPLE_UNIFORM)
    field = G.AnalyticField(cu(gi.c1_scene().packed()))
    ant = cu(gi.antenna_array(16, 16, 0.002))
    f, grad, a, _ = G.geraf_fields(field, xyz)
    f_apr, _, _, _ = G.geraf_fields(field, apr, want_grad=False, want_refl=False)
    f_ant, _, _, _ = G.geraf_fields(field, ant, want_grad=False, want_refl=False)
    alpha, T, w, t_eff, c_ant = G.geraf_blend(f, a, g.n_ray, g.n[2], f_apr, f_ant, wl.sharpness, wl.a_tx)
    # the isotropic point reflector, appended: w = 1, T' = 1, zero normal
    pr = gi.c1_point_reflector(g)
    xyz2 = torch.cat([xyz, cu(pr).reshape(3, 1)], 1).contiguous()
    grad2 = torch.cat([grad, torch.zeros(3, 1, device="cuda")], 1).contiguous()
    w2 = torch.cat([w, torch.ones(1, device="cuda")]).contiguous()
    t2 = torch.cat([t_eff, torch.full((1,), 2.0, device="cuda")]).contiguous()
    b = gi.band(77e9, 81e9, wl.n_f)
    s = G.geraf_render(xyz2, grad2, w2, t2, ant, c_ant, _band(G, b))
    P, M, _, _ = G.geraf_filter(s, ant, _band(G, b), xyz)
    G.geraf_poll_device_error()
    # stage parity on identical inputs
    os_ = oracle.render(host(xyz2), host(grad2), host(w2), host(t2), host(ant), host(c_ant), b)
    assert rel_l2(host(s), os_) < TOL
    oM, oP = oracle.filter_forward(host(s), host(ant), host(xyz), b)
    assert rel_l2(host(P), oP) < TOL
    # all-oracle chain from the same sample points
    sc = gi.c1_scene()
    of, oG, oa = oracle.analytic_fields(sc, host(xyz))
    ofa, _, _ = oracle.analytic_fields(sc, host(apr))
    ofn, _, _ = oracle.analytic_fields(sc, host(ant))
    oal, oT, ow, ote, oca = oracle.blend(of, oa, g.n_ray, g.n[2], ofa, ofn, wl.sharpness, wl.a_tx)
    ox = np.concatenate([host(xyz), pr.reshape(3, 1)], 1)
    os2 = oracle.render(ox, np.concatenate([oG, np.zeros((3, 1))], 1), np.append(ow, 1.0), np.append(ote, 2.0),
                        host(ant), oca, b)
    _, oP2 = oracle.filter_forward(os2, host(ant), host(xyz), b)
    # FP32 SDF rounding enters through exp(s f) with s f up to ~60: looser bound for the whole chain
    assert rel_l2(host(P), oP2) < 1e-4
    assert int(np.argmax(host(P))) == int(np.argmax(oP2))


@pytest.mark.parametrize("method", METHODS)
def test_fmcw_multi_plane_scan(G, oracle, method):
    """The paper's radar read as stepped frequencies (64 chirp samples from
    77 GHz at 70.15 MHz/us, 1.25 Msps) on 8 scanning planes of 6x5 antennas
    around a 10 cm cube at 0.4 m: all four phasor sums against the oracle."""
    rng = np.random.default_rng(21)
    b = gi.fmcw_band()
    ant = gi.multi_plane_array(8, 6, 5, 0.002, 0.4)
    xyz, grad, w, t_eff = _scene_points(rng, 2500, (0.0, 0.0, 0.0), 0.05)
    c_ant = rng.uniform(0.2, 1.0, ant.shape[1]).astype(np.float32)
    band = _band(G, b, method)
    s = G.geraf_render(cu(xyz), cu(grad), cu(w), cu(t_eff), cu(ant), cu(c_ant), band, True)
    G.geraf_poll_device_error()
    assert rel_l2(host(s), oracle.render(xyz, grad, w, t_eff, ant, c_ant, b)) < TOL
    g = gi.complex_normal(rng, (ant.shape[1], b.n_f)).astype(np.complex64)
    d_w, d_t, d_g = G.geraf_render_backward(cu(xyz), cu(grad), cu(w), cu(t_eff), cu(ant), cu(c_ant), band,
                                            torch.as_tensor(g, device="cuda"))
    ow, ot, og = oracle.render_backward(xyz, grad, w, t_eff, ant, c_ant, b, g)
    kt = away_from_clamp_kink(t_eff, c_ant)     # d_t: away from the clamp's kinks
    assert rel_l2(host(d_w), ow) < TOL and rel_l2(host(d_t)[kt], ot[kt]) < TOL and rel_l2(host(d_g), og) < 3 * TOL
    vox = (rng.uniform(-0.05, 0.05, (3, 1500))).astype(np.float32)
    sv = gi.complex_normal(rng, (ant.shape[1], b.n_f)).astype(np.complex64)
    P, M, _, _ = G.geraf_filter(torch.as_tensor(sv, device="cuda"), cu(ant), band, cu(vox))
    oM, oP = oracle.filter_forward(sv, ant, vox, b)
    assert rel_l2(host(M), oM) < TOL
    d_P = rng.standard_normal(vox.shape[1]).astype(np.float32)
    gs = G.geraf_filter_backward(cu(ant), band, cu(vox), M, cu(d_P))
    G.geraf_poll_device_error()
    assert rel_l2(host(gs), oracle.filter_backward(host(M), d_P, ant, vox, b)) < TOL
    if method == 2:
        assert G.geraf_chebyshev_order(cu(xyz), cu(ant), band) > 0


@pytest.mark.parametrize("dist,cheb", [(1.8, True), (2.5, False)])
def test_far_array_split_range_bound(G, oracle, dist, cheb):
    """The Chebyshev kernels form the pair range from coordinates in carrier
    cycles split on a half-cycle grid, exact while every axis difference stays
    below 1024 cycles (about 1.94 m at the 79 GHz band centre); the device plan sends farther
    calls to the per-bin recurrence kernels. A small array `dist` metres in
    front of the cube: at 1.8 m the Chebyshev form runs, at 2.5 m the
    recurrence does, and both match the oracle."""
    rng = np.random.default_rng(21)
    n_pts, n_f = 1500, 128
    xyz, grad, w, t_eff = _scene_points(rng, n_pts)
    ant = gi.antenna_array(6, 5, 0.004, center=(0.01, -0.02, 0.15 - dist))
    c_ant = rng.uniform(0.2, 1.0, ant.shape[1]).astype(np.float32)
    b = gi.band(77e9, 81e9, n_f)
    order = G.geraf_chebyshev_order(cu(xyz), cu(ant), _band(G, b))
    assert (order > 0) == cheb, order
    s = G.geraf_render(cu(xyz), cu(grad), cu(w), cu(t_eff), cu(ant), cu(c_ant), _band(G, b), True)
    G.geraf_poll_device_error()
    assert rel_l2(host(s), oracle.render(xyz, grad, w, t_eff, ant, c_ant, b)) < TOL
    g = gi.complex_normal(rng, (ant.shape[1], n_f)).astype(np.complex64)
    d_w, d_t, d_g = G.geraf_render_backward(cu(xyz), cu(grad), cu(w), cu(t_eff), cu(ant), cu(c_ant),
                                            _band(G, b), torch.as_tensor(g, device="cuda"))
    G.geraf_poll_device_error()
    ow, ot, og = oracle.render_backward(xyz, grad, w, t_eff, ant, c_ant, b, g)
    kt = away_from_clamp_kink(t_eff, c_ant)     # d_t: away from the clamp's kinks
    assert rel_l2(host(d_w), ow) < TOL and rel_l2(host(d_t)[kt], ot[kt]) < TOL and rel_l2(host(d_g), og) < 3 * TOL
    vox = (np.array([0.0, 0.0, 0.15])[:, None] + rng.uniform(-0.05, 0.05, (3, 900))).astype(np.float32)
    sig = torch.as_tensor(oracle.render(xyz, grad, w, t_eff, ant, c_ant, b).astype(np.complex64), device="cuda")
    P, M, _, _ = G.geraf_filter(sig, cu(ant), _band(G, b), cu(vox))
    G.geraf_poll_device_error()
    oM, _ = oracle.filter_forward(host(sig), ant, vox, b)
    assert rel_l2(host(M), oM) < TOL


@pytest.mark.parametrize("wide_first", [True, False])
def test_chebyshev_groups_mixed_orders(G, oracle, wide_first):
    """The Chebyshev kernels expand each split of points (to bins) and each
    group of 2048 points or voxels (to points) over its own range interval with
    its own order. Consecutive chunks of 2048 points here lie in clusters of
    very different range spread (about 44 terms for the wide one, ~8 for the
    compact ones), so the orders differ from group to group and the instance
    chosen by the largest order (K <= 64 with the wide chunk, K <= 24 without)
    runs groups of lower order; 3 x 2048 + 517 points leave a ragged last
    group. Every phasor call against the oracle."""
    rng = np.random.default_rng(31)
    chunks = [((0.0, 0.0, 0.35) if wide_first else (0.0, 0.0, 0.30), 0.25 if wide_first else 0.01, 2048),
              ((0.02, -0.01, 0.12), 0.01, 2048),
              ((-0.03, 0.02, 0.20), 0.015, 2048), ((0.0, 0.04, 0.16), 0.008, 517)]
    parts = [_scene_points(rng, n, c, h) for c, h, n in chunks]
    xyz, grad, w, t_eff = (np.concatenate([p[i] for p in parts], axis=-1) for i in range(4))
    n_f = 128
    ant = gi.antenna_array(9, 8, 0.002)
    c_ant = rng.uniform(0.2, 1.0, ant.shape[1]).astype(np.float32)
    b = gi.band(77e9, 81e9, n_f)
    band = _band(G, b, 2)
    order = G.geraf_chebyshev_order(cu(xyz), cu(ant), band)
    assert order > (32 if wide_first else 0), order
    s = G.geraf_render(cu(xyz), cu(grad), cu(w), cu(t_eff), cu(ant), cu(c_ant), band, True)
    G.geraf_poll_device_error()
    want = oracle.render(xyz, grad, w, t_eff, ant, c_ant, b)
    assert rel_l2(host(s), want) < TOL
    g = gi.complex_normal(rng, (ant.shape[1], n_f)).astype(np.complex64)
    d_w, d_t, d_g = G.geraf_render_backward(cu(xyz), cu(grad), cu(w), cu(t_eff), cu(ant), cu(c_ant), band,
                                            torch.as_tensor(g, device="cuda"))
    G.geraf_poll_device_error()
    ow, ot, og = oracle.render_backward(xyz, grad, w, t_eff, ant, c_ant, b, g)
    kt = away_from_clamp_kink(t_eff, c_ant)     # d_t: away from the clamp's kinks
    assert rel_l2(host(d_w), ow) < TOL and rel_l2(host(d_t)[kt], ot[kt]) < TOL and rel_l2(host(d_g), og) < 3 * TOL
    sig = torch.as_tensor(want.astype(np.complex64), device="cuda")
    P, M, _, _ = G.geraf_filter(sig, cu(ant), band, cu(xyz))
    G.geraf_poll_device_error()
    oM, _ = oracle.filter_forward(host(sig), ant, xyz, b)
    assert rel_l2(host(M), oM) < TOL
    d_P = rng.standard_normal(xyz.shape[1]).astype(np.float32)
    gb = G.geraf_filter_backward(cu(ant), band, cu(xyz), M, cu(d_P))
    G.geraf_poll_device_error()
    assert rel_l2(host(gb), oracle.filter_backward(host(M), d_P, ant, xyz, b)) < TOL


@pytest.mark.parametrize("wide_first", [True, False])
def test_chebyshev_work_orders(G, wide_first):
    """geraf_chebyshev_work against the order rule stated on the host: the
    largest group order (groups of 2048 points, to points) and the largest
    part order (splits of one 128-point record tile here: 72 antennas leave
    one antenna block, so the plan cuts the points into single tiles), the kernel
    instance that follows from it and the mean orders per pair. Parts are
    runs of consecutive records in the brick order (brick_order)."""
    rng = np.random.default_rng(31)
    chunks = [((0.0, 0.0, 0.30), 0.12 if wide_first else 0.01, 2048), ((0.02, -0.01, 0.12), 0.01, 2048),
              ((-0.03, 0.02, 0.20), 0.015, 2048), ((0.0, 0.04, 0.16), 0.008, 517)]
    xyz = np.concatenate([(np.array(c)[:, None] + rng.uniform(-h, h, (3, n))) for c, h, n in chunks],
                         axis=1).astype(np.float32)
    n = xyz.shape[1]
    ant = gi.antenna_array(9, 8, 0.002)
    b = gi.band(77e9, 81e9, 128)
    band = _band(G, b, 2)
    K = G.geraf_chebyshev_order(cu(xyz), cu(ant), band)
    inst_of = lambda km: 24 if km <= 24 else (32 if km <= 32 else 64)
    for to_points, per in ((True, 2048), (False, 128)):
        k0, km, inst, mean = G.geraf_chebyshev_work(cu(xyz), cu(ant), band, to_points)
        assert k0 == K
        xs = xyz[:, brick_order(xyz)]
        host = [_host_order(xs[:, j:j + per], ant, b) for j in range(0, n, per)]
        assert abs(km - max(host)) <= 1 and km <= K, (km, max(host), K)
        assert inst == inst_of(km)
        counts = [min(n, j + per) - j for j in range(0, n, per)]
        # orders run per pair: the part's order rounded up to even (at least
        # 8) in the 24- and 32-order instances, 32 plus blocks of 8 beyond
        # 32 in the 64-order instance
        ex = [min(inst, max(8, (k + 1) // 2 * 2)) if inst <= 32 else max(32, (k + 7) // 8 * 8) for k in host]
        want = sum(c * e for c, e in zip(counts, ex)) / n
        assert abs(mean - want) < 3.0, (mean, want)
        # the brick order can join records of two clusters in one part (a
        # brick's neighbour along the Z-curve), so narrow clusters do not
        # bound the part orders by their own spans
        assert 8.0 <= mean <= inst
    # the recurrence: all zero
    assert G.geraf_chebyshev_work(cu(xyz), cu(ant), _band(G, b, 1), True) == (0, 0, 0, 0.0)


@pytest.mark.parametrize("half", [0.025, 0.05, 0.08, 0.1])
def test_chebyshev_even_order_dispatch(G, oracle, half):
    """Each CTA of the Chebyshev kernels runs its part's order rounded up to
    even (at least 8) as a compile-time loop bound. Random points in cubes
    of half-side 2.5, 5, 8 and 10 cm in front of a 12 x 11 array (132
    antennas: two blocks of antenna records, each with its own plan) put the
    part orders (one 128-point tile x one antenna block to bins, 2048-point
    groups x one antenna block to points) between about 10 and 25, so most of
    the even bodies run; every phasor call against the oracle."""
    rng = np.random.default_rng(41)
    n_pts, n_f = 4099, 128
    xyz, grad, w, t_eff = _scene_points(rng, n_pts, (0.0, 0.0, 0.15), half)
    ant = gi.antenna_array(12, 11, 0.002)
    c_ant = rng.uniform(0.2, 1.0, ant.shape[1]).astype(np.float32)
    b = gi.band(77e9, 81e9, n_f)
    band = _band(G, b, 2)
    assert G.geraf_chebyshev_order(cu(xyz), cu(ant), band) > 0
    s = G.geraf_render(cu(xyz), cu(grad), cu(w), cu(t_eff), cu(ant), cu(c_ant), band, True)
    G.geraf_poll_device_error()
    want = oracle.render(xyz, grad, w, t_eff, ant, c_ant, b)
    assert rel_l2(host(s), want) < TOL
    g = gi.complex_normal(rng, (ant.shape[1], n_f)).astype(np.complex64)
    d_w, d_t, d_g = G.geraf_render_backward(cu(xyz), cu(grad), cu(w), cu(t_eff), cu(ant), cu(c_ant), band,
                                            torch.as_tensor(g, device="cuda"))
    G.geraf_poll_device_error()
    ow, ot, og = oracle.render_backward(xyz, grad, w, t_eff, ant, c_ant, b, g)
    kt = away_from_clamp_kink(t_eff, c_ant)     # d_t: away from the clamp's kinks
    assert rel_l2(host(d_w), ow) < TOL and rel_l2(host(d_t)[kt], ot[kt]) < TOL
    # the directional factor max(2 c^2 - 1, 0) has a kink at c^2 = 1/2, where its
    # gradient in the normal jumps: a pair within rounding of it may take the
    # other side in FP32 than in FP64 (either gradient is correct there), so
    # d_G is compared on the points with no antenna within 1e-4 of the kink
    away = away_from_directional_kink(xyz, grad, ant, 1e-4)
    assert away.mean() > 0.98
    assert rel_l2(host(d_g)[:, away], og[:, away]) < 3 * TOL
    sig = torch.as_tensor(want.astype(np.complex64), device="cuda")
    P, M, _, _ = G.geraf_filter(sig, cu(ant), band, cu(xyz))
    G.geraf_poll_device_error()
    oM, _ = oracle.filter_forward(host(sig), ant, xyz, b)
    assert rel_l2(host(M), oM) < TOL
    d_P = rng.standard_normal(n_pts).astype(np.float32)
    gb = G.geraf_filter_backward(cu(ant), band, cu(xyz), M, cu(d_P))
    G.geraf_poll_device_error()
    assert rel_l2(host(gb), oracle.filter_backward(host(M), d_P, ant, xyz, b)) < TOL


def test_render_antenna_block_plans(G, oracle):
    """With splits of at least 8192 points the to-bins kernels plan each
    (split, 128-antenna block) over its own range interval: 128 x 128 x 40
    ray-ordered stratified samples against the 64 x 64 array (4096 antennas,
    32 blocks) give 80 splits of 8192 points. The oracle computes the signal
    of 48 antennas spread over the blocks; the GPU computes all of them."""
    g = gi.cube_grid((0.0, 0.0, 0.15), 0.10, (128, 128, 40))
    xyz, _ = oracle.sample(g, gi.SAMPLE_STRATIFIED, seed=3, step=0)
    xyz = xyz.astype(np.float32)
    n = xyz.shape[1]
    rng = np.random.default_rng(51)
    grad = rng.standard_normal((3, n)).astype(np.float32)
    w = rng.uniform(0.0, 1.0, n).astype(np.float32)
    t_eff = rng.uniform(0.3, 2.0, n).astype(np.float32)
    ant = gi.antenna_array(64, 64, 0.002)
    c_ant = rng.uniform(0.2, 1.0, ant.shape[1]).astype(np.float32)
    b = gi.band(77e9, 81e9, 128)
    band = _band(G, b, 2)
    s = host(G.geraf_render(cu(xyz), cu(grad), cu(w), cu(t_eff), cu(ant), cu(c_ant), band, True))
    G.geraf_poll_device_error()
    sub = np.sort(rng.choice(ant.shape[1], 48, replace=False))
    want = oracle.render(xyz, grad, w, t_eff, ant[:, sub], c_ant[sub], b)
    assert rel_l2(s[sub], want) < TOL


@pytest.mark.parametrize("n_side,n_pts", [(70, 1501), (143, 257)])
def test_antenna_order_any_input_order(G, oracle, n_side, n_pts):
    """The Chebyshev calls take the antennas in a spatial (Morton) order of
    their positions, so that every block of 128 antenna records is compact,
    and write every output back in the caller's order. A shuffled array gives
    the oracle's sums and the unshuffled call's results, permuted. 70 x 70 =
    4900 antennas sort in shared memory; 143 x 143 = 20 449 (above 16 384) in
    the global scratch buffer."""
    rng = np.random.default_rng(n_side)
    xyz, grad, w, t_eff = _scene_points(rng, n_pts)
    ant0 = gi.antenna_array(n_side, n_side, 0.002)
    perm = rng.permutation(ant0.shape[1])
    ant = np.ascontiguousarray(ant0[:, perm])
    c_ant = rng.uniform(0.2, 1.0, ant.shape[1]).astype(np.float32)
    b = gi.band(77e9, 81e9, 96)
    band = _band(G, b, 2)
    s = host(G.geraf_render(cu(xyz), cu(grad), cu(w), cu(t_eff), cu(ant), cu(c_ant), band, True))
    G.geraf_poll_device_error()
    assert rel_l2(s, oracle.render(xyz, grad, w, t_eff, ant, c_ant, b)) < TOL
    inv = np.argsort(perm)
    s0 = host(G.geraf_render(cu(xyz), cu(grad), cu(w), cu(t_eff), cu(ant0), cu(c_ant[inv]), band, True))
    assert rel_l2(s, s0[perm]) < TOL
    g = gi.complex_normal(rng, (ant.shape[1], b.n_f)).astype(np.complex64)
    d_w, d_t, d_g = G.geraf_render_backward(cu(xyz), cu(grad), cu(w), cu(t_eff), cu(ant), cu(c_ant), band,
                                            torch.as_tensor(g, device="cuda"))
    G.geraf_poll_device_error()
    ow, ot, og = oracle.render_backward(xyz, grad, w, t_eff, ant, c_ant, b, g)
    kt = away_from_clamp_kink(t_eff, c_ant)
    kd = away_from_directional_kink(xyz, grad, ant, 1e-4)
    assert rel_l2(host(d_w), ow) < TOL and rel_l2(host(d_t)[kt], ot[kt]) < TOL
    assert rel_l2(host(d_g)[:, kd], og[:, kd]) < 3 * TOL
    sig = torch.as_tensor(s, device="cuda")
    P, M, _, _ = G.geraf_filter(sig, cu(ant), band, cu(xyz))
    G.geraf_poll_device_error()
    oM, _ = oracle.filter_forward(s, ant, xyz, b)
    assert rel_l2(host(M), oM) < TOL
    d_P = rng.standard_normal(n_pts).astype(np.float32)
    gb = G.geraf_filter_backward(cu(ant), band, cu(xyz), M, cu(d_P))
    G.geraf_poll_device_error()
    assert rel_l2(host(gb), oracle.filter_backward(host(M), d_P, ant, xyz, b)) < TOL
