"""Pins for the oracle's lensless alpha blending: the telescoping closed form of
the NeuS product, the integral definition of alpha (App. B.1) by quadrature,
the transmittance correction against a brute-force march along the real ray
(App. B.2), and the hand-written adjoint against finite differences."""
import numpy as np
from scipy import integrate

import geraf_inputs as gi


def test_monotone_column_telescopes(oracle):
    # plane f = D - z entered from the front: alpha_k > 0, T_k = Phi_k / Phi_0
    s, n_z = 300.0, 40
    z = np.linspace(0.10, 0.20, n_z)
    f = 0.15 - z
    alpha, T, w, t_eff, _ = oracle.blend(f, np.full(n_z, 0.5), 1, n_z, np.array([1.0]), np.zeros(1), s, 2.0)
    Phi = 1.0 / (1.0 + np.exp(-s * f))
    np.testing.assert_allclose(T, Phi / Phi[0], rtol=1e-12)
    np.testing.assert_allclose((T * alpha).sum(), 1.0 - Phi[-1] / Phi[0], rtol=1e-12)
    np.testing.assert_allclose(w, 0.5 * alpha * 2.0, rtol=1e-15)
    assert alpha[-1] == 0.0
    np.testing.assert_allclose(t_eff - T, 1.0 / (1.0 + np.exp(-s)), rtol=1e-15)


def test_exiting_column_has_no_opacity(oracle):
    z = np.linspace(0.1, 0.2, 10)
    alpha, T, *_ = oracle.blend(z - 0.15, np.ones(10), 1, 10, np.zeros(1), np.zeros(1), 200.0, 1.0)
    assert np.all(alpha == 0.0) and np.all(T == 1.0)


def _rho(s, fn, x0, d, u, h=1e-7):
    """Opaque density max(-dPhi/du / Phi, 0) along x0 + u d (App. B.1)."""
    Phi = lambda uu: 1.0 / (1.0 + np.exp(-s * fn(x0 + uu * d)))
    dPhi = (Phi(u + h) - Phi(u - h)) / (2 * h)
    return max(-dPhi / Phi(u), 0.0)


def _sphere_sdf(c, R):
    c = np.asarray(c, np.float64)
    return lambda x: np.linalg.norm(x - c) - R


def test_alpha_equals_integral_on_primary_and_oblique_rays(oracle):
    s = 150.0
    fn = _sphere_sdf((0.0, 0.0, 0.15), 0.03)
    # two points on a primary column (direction +z) entering the sphere
    xa, xb = np.array([0.01, 0.0, 0.115]), np.array([0.01, 0.0, 0.125])
    fa, fb = fn(xa), fn(xb)
    alpha, *_ = oracle.blend(np.array([fa, fb]), np.ones(2), 1, 2, np.zeros(1), np.zeros(1), s, 1.0)
    d = xb - xa
    I = integrate.quad(lambda u: _rho(s, fn, xa, d, u), 0.0, 1.0, epsabs=1e-13, epsrel=1e-11)[0]
    np.testing.assert_allclose(alpha[0], 1.0 - np.exp(-I), rtol=1e-6)
    # oblique ray through the same two SDF levels (App. B.1: alpha is direction free)
    u = np.array([0.3, 0.1, 0.95]); u /= np.linalg.norm(u)
    from scipy.optimize import brentq
    start = np.array([-0.02, 0.0, 0.05])
    ua = brentq(lambda t: fn(start + t * u) - fa, 0.0, 0.1)
    ub = brentq(lambda t: fn(start + t * u) - fb, ua, 0.12)
    I2 = integrate.quad(lambda t: _rho(s, fn, start, u, t), ua, ub, epsabs=1e-13, epsrel=1e-11)[0]
    np.testing.assert_allclose(alpha[0], 1.0 - np.exp(-I2), rtol=1e-6)


def test_lensless_transmittance_matches_real_ray_march(oracle):
    """App. B.2: T along the real ray (antenna -> point) is the primary-ray T
    shifted by the origin sigmoid-SDF values: T' = T + Phi(x_apr) - Phi(x_ant).
    Checked near the first surface, where the correction is first order."""
    s = 60.0
    fn = _sphere_sdf((0.0, 0.0, 0.08), 0.03)
    x_apr = np.array([0.004, 0.0, 0.0])
    x_ant = np.array([0.03, 0.012, 0.0])
    n_z = 4000
    z = np.linspace(0.0, 0.049, n_z)
    col = np.stack([np.full(n_z, x_apr[0]), np.full(n_z, x_apr[1]), z])
    f = np.array([fn(col[:, k]) for k in range(n_z)])
    Phi = lambda y: 1.0 / (1.0 + np.exp(-s * fn(y)))
    _, T, _, t_eff, c_ant = oracle.blend(f, np.ones(n_z), 1, n_z, np.array([fn(x_apr)]),
                                         np.array([fn(x_ant)]), s, 1.0)
    corr = Phi(x_apr) - Phi(x_ant)
    assert abs(corr) > 5e-3
    for k in (n_z // 4, n_z // 3, n_z // 2):
        x = col[:, k]
        d = x - x_ant
        I = integrate.quad(lambda t: _rho(s, fn, x_ant, d, t), 0.0, 1.0, epsabs=1e-12, epsrel=1e-10,
                           limit=200)[0]
        T_real = np.exp(-I)
        T_lensless = t_eff[k] - c_ant[0]
        assert T[k] > 0.8
        assert abs(T_real - T_lensless) < 0.2 * abs(corr)
        # the opposite sign of the correction misses by about twice its size
        assert abs(T_real - (T[k] - corr)) > 1.5 * abs(corr)


def test_blend_backward_matches_finite_differences(oracle):
    rng = np.random.default_rng(2)
    n_ray, n_z, s, atx = 3, 9, 80.0, 1.7
    f = np.sort(rng.uniform(-0.03, 0.03, (n_z, n_ray)), axis=0)[::-1].reshape(-1).copy()
    f[5] += 0.01  # a non-monotone step somewhere
    a = rng.uniform(0.2, 1.0, n_z * n_ray)
    dw, dt = rng.standard_normal(n_z * n_ray), rng.standard_normal(n_z * n_ray)

    def L(f_, a_, s_, atx_):
        _, _, w, t_eff, _ = oracle.blend(f_, a_, n_ray, n_z, np.zeros(n_ray), np.zeros(1), s_, atx_)
        return (w * dw).sum() + (t_eff * dt).sum()

    d_f, d_a, d_s, d_atx = oracle.blend_backward(f, a, n_ray, n_z, s, atx, dw, dt)
    h = 1e-7
    for j in range(f.size):
        e = np.zeros_like(f); e[j] = h
        np.testing.assert_allclose(d_f[j], (L(f + e, a, s, atx) - L(f - e, a, s, atx)) / (2 * h),
                                   rtol=1e-5, atol=1e-6)
        np.testing.assert_allclose(d_a[j], (L(f, a + e, s, atx) - L(f, a - e, s, atx)) / (2 * h),
                                   rtol=1e-6, atol=1e-8)
    np.testing.assert_allclose(d_s, (L(f, a, s + 1e-4, atx) - L(f, a, s - 1e-4, atx)) / 2e-4, rtol=1e-5)
    np.testing.assert_allclose(d_atx, (L(f, a, s, atx + h) - L(f, a, s, atx - h)) / (2 * h), rtol=1e-6)
