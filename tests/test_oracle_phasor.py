"""Pins for the oracle's phasor sums (signal tracing, matched filter, adjoints).

Independent evidence used: a numerically simulated FMCW dechirp of a delayed
chirp (section 3, Eq. fmcw), the paper's printed radar constants and range
resolution (App. C), the exact phase cancellation of the matched filter at a
true reflector, resolution formulas, linearity, a pure-Python brute force that
forms the reflection vectors explicitly, adjoint identities and finite
differences."""
import cmath
import math
import os

import numpy as np
import pytest

import geraf_inputs as gi

C = 299792458.0
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _radar_constants():
    out = {}
    for line in open(os.path.join(GOLDEN, "radar_constants.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


def _iso_point(x):
    """One isotropic point (zero normal) with w = 1 and lensless T = 1."""
    xyz = np.asarray(x, np.float64).reshape(3, 1)
    return xyz, np.zeros((3, 1)), np.ones(1), np.full(1, 2.0)


def test_paper_radar_constants_are_consistent():
    rc = _radar_constants()
    df = rc["chirp_slope_hz_per_s"] / rc["sample_rate_sps"]          # frequency step per ADC sample
    B = df * rc["adc_samples"]
    assert abs(B - rc["usable_bandwidth_hz"]) / rc["usable_bandwidth_hz"] < 2e-3
    assert abs(C / (2 * B) - rc["range_resolution_m"]) < 0.005


def test_render_matches_simulated_fmcw_dechirp(oracle):
    """Eq. fmcw: mixing the received (delayed) chirp with the conjugate of the
    transmitted one. The stepped-frequency model uses f_n = f0 + k t_n."""
    rc = _radar_constants()
    k, fs, N, f0 = rc["chirp_slope_hz_per_s"], rc["sample_rate_sps"], int(rc["adc_samples"]), rc["start_frequency_hz"]
    band = gi.Band(f0=f0, df=k / fs, n_f=N)
    ant = np.array([[0.004, -0.01], [0.0, 0.006], [0.0, 0.0]])
    pt = np.array([0.013, -0.021, 0.31])
    xyz, G, w, t_eff = _iso_point(pt)
    s = oracle.render(xyz, G, w, t_eff, ant, np.ones(2), band)
    t = np.arange(N) / fs
    for i in range(2):
        R = np.linalg.norm(pt - ant[:, i])
        tau = 2 * R / C
        phase_tx = lambda tt: 2 * np.pi * (f0 * tt + 0.5 * k * tt * tt)
        beat = np.exp(1j * (phase_tx(t - tau) - phase_tx(t)))       # rx * conj(tx)
        amp = 1.0 / (4 * np.pi * R) ** 2                              # one-way-squared spreading
        np.testing.assert_allclose(s[i], amp * beat, rtol=2e-3, atol=0)


def _grid_centres(grid):
    nx, ny, nz = grid.n
    ii = np.arange(grid.n_pts)
    ix, iy, iz = ii % nx, (ii // nx) % ny, ii // (nx * ny)
    return np.stack([np.float64(grid.lo[d]) + (np.stack([ix, iy, iz])[d] + 0.5) * np.float64(grid.pitch[d])
                     for d in range(3)])


def test_filter_peaks_at_reflector_with_exact_value(oracle):
    band = gi.band(77e9, 81e9, 16)
    ant = gi.antenna_array(6, 6, 0.002).astype(np.float64)
    grid = gi.cube_grid((0.0, 0.0, 0.15), 0.06, (7, 7, 9))
    vox = _grid_centres(grid)
    j = 4 * 49 + 3 * 7 + 2
    xyz, G, w, t_eff = _iso_point(vox[:, j])
    s = oracle.render(xyz, G, w, t_eff, ant, np.ones(ant.shape[1]), band)
    M, P = oracle.filter_forward(s, ant, vox, band)
    assert int(np.argmax(P)) == j
    r = np.linalg.norm(vox[:, j][:, None] - ant, axis=0)
    exact = band.n_f * (1.0 / (4 * np.pi * r) ** 2).sum()          # every phase cancels
    np.testing.assert_allclose(P[j], exact, rtol=1e-12)
    assert abs(M[j].imag) < 1e-12 * exact


def test_filter_range_resolution_matches_paper(oracle):
    """App. C: 3.59 GHz of sweep gives 0.04 m range resolution. The first
    null of the matched-filter range profile of one reflector sits c/(2B) away."""
    rc = _radar_constants()
    band = gi.Band(f0=rc["start_frequency_hz"], df=rc["chirp_slope_hz_per_s"] / rc["sample_rate_sps"],
                   n_f=int(rc["adc_samples"]))
    ant = np.zeros((3, 1))
    z0 = 0.4
    xyz, G, w, t_eff = _iso_point([0.0, 0.0, z0])
    s = oracle.render(xyz, G, w, t_eff, ant, np.ones(1), band)
    dz = np.linspace(0.0, 0.06, 1201)
    vox = np.stack([np.zeros_like(dz), np.zeros_like(dz), z0 + dz])
    _, P = oracle.filter_forward(s, ant, vox, band)
    first_null = dz[np.argmax(np.diff(P) > 0)]           # P decreases until the first null
    assert abs(first_null - rc["range_resolution_m"]) < 0.0025
    assert abs(first_null - C / (2 * band.n_f * band.df)) < 1e-4


def test_filter_cross_range_resolution(oracle):
    band = gi.band(77e9, 81e9, 8)
    n, pitch, R = 16, 0.002, 0.15
    ant = gi.antenna_array(n, n, pitch).astype(np.float64)
    xyz, G, w, t_eff = _iso_point([0.0, 0.0, R])
    s = oracle.render(xyz, G, w, t_eff, ant, np.ones(ant.shape[1]), band)
    dx = np.linspace(0.0, 0.03, 601)
    vox = np.stack([dx, np.zeros_like(dx), np.full_like(dx, R)])
    _, P = oracle.filter_forward(s, ant, vox, band)
    first_null = dx[np.argmax(np.diff(P) > 0)]
    lam = C / (band.f0 + 0.5 * (band.n_f - 1) * band.df)
    L = n * pitch
    predicted = lam * R / (2 * L)
    assert abs(first_null - predicted) / predicted < 0.15


def test_linearity_and_superposition(oracle):
    rng = np.random.default_rng(0)
    band = gi.band(77e9, 81e9, 5)
    ant = gi.antenna_array(3, 2, 0.002).astype(np.float64)
    xyz = np.array([0, 0, 0.15])[:, None] + rng.uniform(-0.03, 0.03, (3, 20))
    G = rng.standard_normal((3, 20))
    t_eff = rng.uniform(0.5, 1.8, 20)
    c_ant = rng.uniform(0.6, 1.0, ant.shape[1])
    w1, w2 = rng.uniform(0, 1, 20), rng.uniform(0, 1, 20)
    s1 = oracle.render(xyz, G, w1, t_eff, ant, c_ant, band)
    s2 = oracle.render(xyz, G, w2, t_eff, ant, c_ant, band)
    s12 = oracle.render(xyz, G, 2.5 * w1 + w2, t_eff, ant, c_ant, band)
    np.testing.assert_allclose(s12, 2.5 * s1 + s2, rtol=1e-12, atol=1e-12 * np.abs(s12).max())
    vox = np.array([0, 0, 0.15])[:, None] + rng.uniform(-0.03, 0.03, (3, 11))
    M1, P1 = oracle.filter_forward(s1, ant, vox, band)
    M2, P2 = oracle.filter_forward((-1.5 + 2j) * s1, ant, vox, band)
    np.testing.assert_allclose(P2, 2.5 * P1, rtol=1e-12)
    np.testing.assert_allclose(M2, (-1.5 + 2j) * M1, rtol=1e-12)


def _brute_render(xyz, G, w, t_eff, ant, c_ant, band):
    """Term-by-term restatement with the reflection vectors formed explicitly."""
    n_ant, n_pts = ant.shape[1], xyz.shape[1]
    s = [[0j] * band.n_f for _ in range(n_ant)]
    for i in range(n_ant):
        for j in range(n_pts):
            d = [xyz[k][j] - ant[k][i] for k in range(3)]
            r = math.sqrt(sum(v * v for v in d))
            w_i = [v / r for v in d]
            gn = math.sqrt(sum(v * v for v in G[:, j]))
            if gn > 0:
                nrm = [v / gn for v in G[:, j]]
                ndot = sum(a * b for a, b in zip(nrm, w_i))
                w_o = [a - 2 * ndot * b for a, b in zip(w_i, nrm)]
                D = max(sum(a * -b for a, b in zip(w_o, w_i)), 0.0)
            else:
                D = 1.0
            T = min(max(t_eff[j] - c_ant[i], 0.0), 1.0)
            A = w[j] * T * T * D / (4 * math.pi * r) ** 2
            for n in range(band.n_f):
                f = band.f0 + n * band.df
                s[i][n] += A * cmath.exp(-2j * math.pi * f * 2 * r / C)
    return np.array(s)


def test_render_equals_brute_force_on_tiny_grid(oracle):
    rng = np.random.default_rng(4)
    band = gi.band(77e9, 81e9, 3)
    ant = gi.antenna_array(2, 2, 0.002).astype(np.float64)
    g = gi.cube_grid((0, 0, 0.12), 0.02, (2, 2, 2))
    xyz = _grid_centres(g)
    G = rng.standard_normal((3, 8)); G[:, 3] = 0.0
    w, t_eff, c_ant = rng.uniform(0, 1, 8), rng.uniform(0.2, 1.9, 8), rng.uniform(0.5, 1.0, 4)
    s = oracle.render(xyz, G, w, t_eff, ant, c_ant, band)
    np.testing.assert_allclose(s, _brute_render(xyz, G, w, t_eff, ant, c_ant, band), rtol=1e-13,
                               atol=1e-14 * np.abs(s).max())


def test_directional_factor_special_cases(oracle):
    band = gi.band(77e9, 81e9, 2)
    ant = np.zeros((3, 1))
    r = 0.1
    xyz = np.array([[0.0], [0.0], [r]])
    base = oracle.render(xyz, np.zeros((3, 1)), np.ones(1), np.full(1, 2.0), ant, np.ones(1), band)
    for normal, want in [((0, 0, -1), 1.0), ((0, 0, 1), 1.0), ((1, 0, 0), 0.0),
                         ((1, 0, 1), 0.0), ((np.sin(0.3), 0, np.cos(0.3)), np.cos(0.6))]:
        s = oracle.render(xyz, np.array(normal, float).reshape(3, 1), np.ones(1), np.full(1, 2.0),
                          ant, np.ones(1), band)
        np.testing.assert_allclose(s, want * base, rtol=1e-12, atol=1e-15 * abs(base).max())


def test_adjoint_identities(oracle):
    rng = np.random.default_rng(5)
    band = gi.band(77e9, 81e9, 7)
    ant = gi.antenna_array(3, 3, 0.003).astype(np.float64)
    n = 30
    xyz = np.array([0, 0, 0.15])[:, None] + rng.uniform(-0.04, 0.04, (3, n))
    G = rng.standard_normal((3, n))
    t_eff, c_ant = rng.uniform(0.2, 1.9, n), rng.uniform(0.5, 1.0, 9)
    w = rng.uniform(0, 1, n)
    g = gi.complex_normal(rng, (9, band.n_f))
    s = oracle.render(xyz, G, w, t_eff, ant, c_ant, band)
    d_w, _, _ = oracle.render_backward(xyz, G, w, t_eff, ant, c_ant, band, g)
    lhs = np.real(np.vdot(g, s))                      # <s, g> as a real inner product
    np.testing.assert_allclose(lhs, (w * d_w).sum(), rtol=1e-11)
    # filter's linear map M(s) and the transpose used by its backward
    vox = np.array([0, 0, 0.15])[:, None] + rng.uniform(-0.04, 0.04, (3, 13))
    cvec = gi.complex_normal(rng, 13)
    M, _ = oracle.filter_forward(s, ant, vox, band)
    gs = oracle.filter_backward(cvec, np.abs(cvec), ant, vox, band)   # dP * M/|M| = c
    np.testing.assert_allclose(np.real(np.vdot(cvec, M)), np.real(np.vdot(gs, s)), rtol=1e-11)


def test_render_backward_matches_finite_differences(oracle):
    rng = np.random.default_rng(6)
    band = gi.band(77e9, 81e9, 6)
    ant = gi.antenna_array(2, 3, 0.004).astype(np.float64)
    n = 5
    xyz = np.array([0, 0, 0.13])[:, None] + rng.uniform(-0.03, 0.03, (3, n))
    G = rng.standard_normal((3, n)) + np.array([0, 0, -2.0])[:, None]
    t_eff, c_ant = rng.uniform(1.05, 1.6, n), rng.uniform(0.7, 0.95, 6)
    w = rng.uniform(0.1, 1, n)
    g = gi.complex_normal(rng, (6, band.n_f))
    L = lambda w_, t_, G_: np.real(np.vdot(g, oracle.render(xyz, G_, w_, t_, ant, c_ant, band)))
    d_w, d_t, d_G = oracle.render_backward(xyz, G, w, t_eff, ant, c_ant, band, g)
    h = 1e-6
    for j in range(n):
        e = np.zeros(n); e[j] = h
        np.testing.assert_allclose(d_t[j], (L(w, t_eff + e, G) - L(w, t_eff - e, G)) / (2 * h),
                                   rtol=1e-6, atol=1e-9 * abs(d_t).max())
        for d in range(3):
            E = np.zeros((3, n)); E[d, j] = h
            np.testing.assert_allclose(d_G[d, j], (L(w, t_eff, G + E) - L(w, t_eff, G - E)) / (2 * h),
                                       rtol=1e-5, atol=1e-8 * abs(d_G).max())


def test_render_backward_clamp_slope_decided_on_the_exact_difference(oracle):
    """The lensless transmittance T' = clamp(t_eff - c_ant, 0, 1) (section 6,
    App. B.2) has kinks at 0 and 1. The oracle takes the side of each kink
    from the exact FP64 difference of its (FP32-valued) inputs: pairs 2^-24 or
    2^-25 away from a kink, where FP32 rounding of the difference would land
    on the kink itself, get the derivative of the side they lie on (central
    differences with a step well inside that side), and 0 outside [0, 1]."""
    band = gi.band(77e9, 81e9, 5)
    ant = np.zeros((3, 1))
    xyz = np.array([[0.004], [-0.003], [0.13]])
    G = np.zeros((3, 1))                                   # isotropic: D = 1
    w = np.array([0.7])
    g = gi.complex_normal(np.random.default_rng(3), (1, band.n_f))
    cases = [(1.5, 0.5 - 2.0 ** -25, False),               # t - c = 1 + 2^-25: clamped at 1
             (1.5, 0.5 + 2.0 ** -24, True),                # 1 - 2^-24: inside
             (0.5, 0.5 + 2.0 ** -24, False),               # -2^-24: clamped at 0
             (0.5, 0.5 - 2.0 ** -25, True)]                # 2^-25: inside
    for t0, c0, inside in cases:
        t_eff, c_ant = np.array([t0]), np.array([c0])
        assert np.float32(t0) == t0 and np.float32(c0) == c0
        L = lambda t_: np.real(np.vdot(g, oracle.render(xyz, G, w, t_, ant, c_ant, band)))
        _, d_t, _ = oracle.render_backward(xyz, G, w, t_eff, ant, c_ant, band, g)
        h = 2.0 ** -32
        fd = (L(t_eff + h) - L(t_eff - h)) / (2 * h)
        if inside:
            assert d_t[0] != 0.0
            np.testing.assert_allclose(d_t[0], fd, rtol=1e-4)
        else:
            assert d_t[0] == 0.0 and fd == 0.0


def test_filter_backward_matches_finite_differences(oracle):
    rng = np.random.default_rng(7)
    band = gi.band(77e9, 81e9, 4)
    ant = gi.antenna_array(2, 2, 0.003).astype(np.float64)
    vox = np.array([0, 0, 0.15])[:, None] + rng.uniform(-0.04, 0.04, (3, 9))
    s = gi.complex_normal(rng, (4, band.n_f))
    dP = rng.standard_normal(9)
    M, P = oracle.filter_forward(s, ant, vox, band)
    g = oracle.filter_backward(M, dP, ant, vox, band)
    L = lambda s_: (oracle.filter_forward(s_, ant, vox, band)[1] * dP).sum()
    h = 1e-7
    for i in range(4):
        for n in range(band.n_f):
            E = np.zeros_like(s); E[i, n] = h
            np.testing.assert_allclose(g[i, n].real, (L(s + E) - L(s - E)) / (2 * h), rtol=1e-6, atol=1e-9)
            np.testing.assert_allclose(g[i, n].imag, (L(s + 1j * E) - L(s - 1j * E)) / (2 * h),
                                       rtol=1e-6, atol=1e-9)


def test_flat_plate_specular_response(oracle):
    """A plate z = D facing the array: the antenna under the plate centre sees
    a phase slope of -4 pi D df / c per frequency step, and the strongest
    return; normal incidence gives directional factor 1."""
    D = 0.14
    scene = gi.Scene([gi.Prim(gi.PRIM_HALFSPACE, 1.0, (0.0, 0.0, D), (0.0, 0.0, -1.0))])
    grid = gi.cube_grid((0.0, 0.0, D), 0.02, (40, 40, 40))   # lambda/8 lateral sampling
    xyz, apr = oracle.sample(grid, gi.SAMPLE_UNIFORM)
    f, G, a = oracle.analytic_fields(scene, xyz)
    fa, _, _ = oracle.analytic_fields(scene, apr)
    ant = gi.antenna_array(5, 1, 0.004)
    fant, _, _ = oracle.analytic_fields(scene, ant)
    s_sharp = 2.0 / grid.pitch[2]
    alpha, T, w, t_eff, c_ant = oracle.blend(f, a, grid.n_ray, grid.n[2], fa, fant, s_sharp, 1.0)
    band = gi.band(77e9, 81e9, 32)
    s = oracle.render(xyz, G, w, t_eff, ant, c_ant, band)
    centre = 2
    slope = np.angle((s[centre, 1:] * np.conj(s[centre, :-1])).sum())
    np.testing.assert_allclose(slope, -4 * np.pi * D * band.df / C, rtol=0.02)
    mags = np.abs(s).sum(1)
    assert int(np.argmax(mags)) == centre


def test_dynamic_mask_cases(oracle):
    """Each case of the masking rule, and the masked loss against the plain
    loss on the kept voxels only."""
    p_ref, hi, lo = 10.0, 0.5, 0.1
    P = np.array([0.5, 0.5, 6.0, 0.5, 0.99, 1.0])
    H = np.array([0.0, 5.0, 9.0, 4.99, 7.0, 7.0])
    m, H2 = oracle.dynamic_mask(P, H, p_ref, hi, lo)
    # never high -> kept; high before and low now -> dropped; high now -> kept;
    # just below the high threshold -> kept; just below / at the low threshold
    np.testing.assert_array_equal(m, [1, 0, 1, 1, 0, 1])
    np.testing.assert_array_equal(H2, [0.5, 5.0, 9.0, 4.99, 7.0, 7.0])
    target = np.array([1.0, 2.0, 3.0, 4.0, 5.0, 6.0])
    L, dP = oracle.heatmap_loss(P, target, m)
    keep = m > 0
    L_keep, dP_keep = oracle.heatmap_loss(P[keep], target[keep])
    assert abs(L - L_keep) < 1e-12
    np.testing.assert_array_equal(dP[~keep], 0.0)
    np.testing.assert_allclose(dP[keep], dP_keep)


def test_fmcw_band_and_multi_plane_scan_geometry():
    """The chirp read as stepped frequencies reproduces the paper's radar
    (App. C): 56.12 MHz per ADC sample, 3.59 GHz over 64 samples, 4 cm range
    resolution; scanning planes sit on a circle around the object, evenly
    spaced, each facing it."""
    rc = _radar_constants()
    b = gi.fmcw_band()
    assert b.f0 == rc["start_frequency_hz"] and b.n_f == rc["adc_samples"]
    np.testing.assert_allclose(b.df, rc["chirp_slope_hz_per_s"] / rc["sample_rate_sps"])
    np.testing.assert_allclose(b.n_f * b.df, rc["usable_bandwidth_hz"], rtol=2e-3)
    np.testing.assert_allclose(299792458.0 / (2 * b.n_f * b.df), rc["range_resolution_m"], rtol=0.05)
    n_planes, nx, ny, pitch, radius = 8, 5, 3, 0.002, 0.4
    ctr = np.array([0.0, 0.0, 0.0])
    A = gi.multi_plane_array(n_planes, nx, ny, pitch, radius, ctr).astype(np.float64)
    assert A.shape == (3, n_planes * nx * ny)
    P = A.reshape(3, n_planes, nx * ny)
    mid = P.mean(2)                                               # plane centres
    np.testing.assert_allclose(np.linalg.norm(mid[[0, 2]], axis=0), radius, rtol=1e-6)
    ang = np.unwrap(np.arctan2(mid[0], mid[2]))
    np.testing.assert_allclose(np.diff(ang), 2 * np.pi / n_planes, atol=1e-6)
    for m in range(n_planes):
        d = P[:, m] - mid[:, m:m + 1]
        nrm = -mid[:, m] / np.linalg.norm(mid[:, m])
        np.testing.assert_allclose(d.T @ nrm, 0.0, atol=1e-7)     # the plane faces the centre
        np.testing.assert_allclose(np.sort(np.linalg.norm(d[:, :1] - d, axis=0))[1], pitch, rtol=1e-5)
