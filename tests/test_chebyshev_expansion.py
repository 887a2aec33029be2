"""The mathematics the Chebyshev phasor kernels rest on, checked on the host
(no GPU): the Jacobi-Anger expansion of the bin phase, the order rule
(smallest K whose Bessel tail sum_{k >= K} 2 |J_k(a)| is at most 1e-7, below the
FP32 rounding of the sums), the factorisation of a bin's phase about the
band's centre and an antenna's own range centre, and the range interval of a
part (each antenna's nearest point of the box and farthest corner).

The kernels expand exp(-j a x), |x| <= 1, a = 2 pi m (df / f_c) dr with m the
bin's offset from the band's centre f_c (negative below it) and R, dr in carrier
cycles, as sum_k eps_k (-j)^k J_k(a) T_k(x) (eps_0 = 1, eps_k = 2), truncated
at the order rule; each CTA may run more orders than its part's K (its K
rounded up to even, at least 8), which only adds the series' own next terms.
Bessel values here come from scipy, independent of the device's Miller
recurrence."""
import numpy as np
import pytest

special = pytest.importorskip("scipy.special")

C = 299792458.0


TAIL = 1e-7


def order_rule(a, eps=TAIL, kmax=64):
    J = np.abs(special.jv(np.arange(kmax + 8), a))
    tail = np.cumsum((2 * J)[::-1])[::-1]            # tail[k] = sum_{m >= k} 2 |J_m(a)|
    above = np.nonzero(tail > eps)[0]
    return max(int(above[-1]) + 1, 2) if above.size else 2


def series(a, x, K):
    k = np.arange(K)
    eps = np.where(k == 0, 1.0, 2.0)
    coef = eps * (-1j) ** k * special.jv(k, a)      # [K]
    T = np.cos(np.outer(np.arccos(np.clip(x, -1, 1)), k))   # T_k(x) = cos(k arccos x)
    return T @ coef


@pytest.mark.parametrize("a", [0.0, 0.5, 3.0, 9.7, 21.4, 38.0, -0.5, -9.7, -21.4])
def test_truncation_at_the_order_rule(a):
    """|sum_{k < K} ... - exp(-j a x)| <= the tail bound (1e-7) on a dense x
    grid, for bins on both sides of the band's centre (negative a, order
    rule on |a|), and running more orders (the even-rounded count) never does
    worse."""
    x = np.linspace(-1.0, 1.0, 2001)
    K = order_rule(abs(a))
    err = np.abs(series(a, x, K) - np.exp(-1j * a * x)).max()
    assert err <= TAIL + 1e-13
    Ke = max(8, (K + 1) // 2 * 2)
    err_e = np.abs(series(a, x, min(Ke + 2, 70)) - np.exp(-1j * a * x)).max()
    assert err_e <= err + 1e-13


def test_negative_argument_is_the_conjugate_power():
    """J_k(-a) = (-1)^k J_k(a): the table entry of a bin below the band's
    centre, eps_k (-j)^k J_k(-a), equals eps_k j^k J_k(|a|) (the device
    computes J_k of |a| and takes the power of +j)."""
    k = np.arange(40)
    for a in (0.3, 4.2, 17.9, 33.3):
        lhs = (-1j) ** k * special.jv(k, -a)
        rhs = (1j) ** k * special.jv(k, a)
        np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-15)


def test_bin_phase_factorisation_about_the_centres():
    """exp(-j 2 pi f_n 2 r / c) = exp(-j 2 pi R) exp(-j 2 pi m Kc r_c)
    sum_k eps_k (-j)^k J_k(a_m) T_k(x) to the tail bound, with K0 = 2 f_c / c,
    R = K0 r, Kc = df / f_c, m = n - (n_f - 1) / 2, x = (R - r_c) / dr and
    a_m = 2 pi m Kc dr: a 77-81 GHz band of 256 bins, ranges of one antenna
    over a 2 cm interval at 0.3 m, the order from the largest |a_m|."""
    f0, f1, n_f = 77e9, 81e9, 256
    df = (f1 - f0) / (n_f - 1)
    fc = f0 + 0.5 * (n_f - 1) * df
    K0, Kc = 2 * fc / C, df / fc
    rng = np.random.default_rng(3)
    r = rng.uniform(0.29, 0.31, 300)                 # metres
    R = K0 * r                                       # cycles
    r_c = 0.5 * (R.min() + R.max())
    dr = 0.5 * (R.max() - R.min()) * 1.001
    x = (R - r_c) / dr
    m = np.arange(n_f) - 0.5 * (n_f - 1)
    a = 2 * np.pi * m * Kc * dr
    K = order_rule(np.abs(a).max())
    assert K <= 40
    k = np.arange(K)
    epsk = np.where(k == 0, 1.0, 2.0)
    B = epsk[None, :] * (-1j) ** k[None, :] * special.jv(k[None, :], a[:, None])      # [n_f, K]
    T = np.cos(np.outer(np.arccos(x), k))                                                # [pts, K]
    got = (np.exp(-2j * np.pi * R)[:, None] * np.exp(-2j * np.pi * m * Kc * r_c)[None, :]
           * (T @ B.T))
    f = f0 + df * np.arange(n_f)
    want = np.exp(-2j * np.pi * np.outer(2 * r / C, f))
    assert np.abs(got - want).max() < 2e-7


def test_order_follows_span_times_spread():
    """K depends on the largest argument pi (n_f - 1) (2 df / c) dr only (dr
    in metres): the 4 GHz span over a 16 cm range spread needs about 21
    orders, a 3-4 cm spread about 12, whatever the bin count."""
    span = 4e9
    for n_f in (64, 128, 1024):
        df = span / (n_f - 1)
        a16 = np.pi * (n_f - 1) * (2 * df / C) * 0.08
        a4 = np.pi * (n_f - 1) * (2 * df / C) * 0.02
        assert 18 <= order_rule(a16) <= 26
        assert 9 <= order_rule(a4) <= 15


def test_part_interval_contains_every_pair_range():
    """Each antenna's interval of a part is [nearest point of the box,
    farthest corner]; every (point, antenna) range lies inside it, so with
    r_c the interval's midpoint and dr the largest half span over the part's
    antennas every x = (r - r_c) / dr lies in [-1, 1]; the bound is tight to
    the box (a brute-force check on random parts)."""
    rng = np.random.default_rng(5)
    for _ in range(50):
        c = rng.uniform(-0.05, 0.05, 3) + np.array([0.0, 0.0, 0.15])
        h = rng.uniform(0.001, 0.05, 3)
        pts = c[:, None] + rng.uniform(-1, 1, (3, 400)) * h[:, None]
        ant = rng.uniform(-0.07, 0.07, (3, 64))
        ant[2] = rng.uniform(-0.01, 0.01, 64)
        lo, hi = pts.min(1), pts.max(1)
        near = np.sqrt((np.maximum(np.maximum(lo[:, None] - ant, ant - hi[:, None]), 0.0) ** 2).sum(0))
        far = np.sqrt((np.maximum(np.abs(ant - lo[:, None]), np.abs(hi[:, None] - ant)) ** 2).sum(0))
        r = np.sqrt(((pts[:, :, None] - ant[:, None, :]) ** 2).sum(0))          # [pts, ant]
        assert (near[None, :] <= r + 1e-15).all() and (r <= far[None, :] + 1e-15).all()
        r_c, dr = 0.5 * (near + far), (0.5 * (far - near)).max()
        assert np.abs((r - r_c[None, :]) / dr).max() <= 1 + 1e-12
        # the per-antenna half span is never wider than the block-shared one
        assert dr <= 0.5 * (far.max() - near.min()) + 1e-15
        # tight for the box: the box's own corners reach each antenna's bounds
        corners = np.stack(np.meshgrid(*zip(lo, hi), indexing="ij"), 0).reshape(3, -1)
        rc = np.sqrt(((corners[:, :, None] - ant[:, None, :]) ** 2).sum(0))
        assert np.abs(rc.max(0) - far).max() < 1e-12
