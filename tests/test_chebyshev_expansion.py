"""The mathematics the Chebyshev phasor kernels rest on, checked on the host
(no GPU): the Jacobi-Anger expansion of the bin phase, the order rule
(smallest K whose Bessel tail sum_{k >= K} 2 |J_k(a)| is at most 1e-7, below the
FP32 rounding of the sums), and the
range interval of a part (nearest point of its bounding box, farthest corner).

The kernels expand exp(-j a x), |x| <= 1, a = 2 pi n (2 df / c) dr, as
sum_k eps_k (-j)^k J_k(a) T_k(x) (eps_0 = 1, eps_k = 2), truncated at the order
rule; each CTA may run more orders than its part's K (its K rounded up to
even, at least 8), which only adds the series' own next terms. Bessel values
here come from scipy, independent of the device's Miller recurrence."""
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


@pytest.mark.parametrize("a", [0.0, 0.5, 3.0, 9.7, 21.4, 38.0])
def test_truncation_at_the_order_rule(a):
    """|sum_{k < K} ... - exp(-j a x)| <= the tail bound (1e-7) on a dense x
    grid, and running more orders (the even-rounded count) never does worse."""
    x = np.linspace(-1.0, 1.0, 2001)
    K = order_rule(a)
    err = np.abs(series(a, x, K) - np.exp(-1j * a * x)).max()
    assert err <= TAIL + 1e-13
    Ke = max(8, (K + 1) // 2 * 2)
    err_e = np.abs(series(a, x, min(Ke + 2, 70)) - np.exp(-1j * a * x)).max()
    assert err_e <= err + 1e-13


def test_order_follows_span_times_spread():
    """K depends on a_max = 2 pi (n_f - 1) (2 df / c) dr only: the 4 GHz span
    over a 16 cm range spread (the C2 volume against the 64 x 64 array) needs
    about 32 orders, a 3-4 cm slab about 20, whatever the bin count."""
    span = 4e9
    for n_f in (64, 128, 1024):
        df = span / (n_f - 1)
        a16 = 2 * np.pi * (n_f - 1) * (2 * df / C) * 0.08
        a4 = 2 * np.pi * (n_f - 1) * (2 * df / C) * 0.02
        assert 28 <= order_rule(a16) <= 36
        assert 14 <= order_rule(a4) <= 24


def test_part_interval_contains_every_pair_range():
    """The interval of a part is [nearest point of its box, farthest corner]
    over its antennas; every (point, antenna) range of the part lies inside,
    and the bound is tight to the box (a brute-force check on random parts)."""
    rng = np.random.default_rng(5)
    for _ in range(50):
        c = rng.uniform(-0.05, 0.05, 3) + np.array([0.0, 0.0, 0.15])
        h = rng.uniform(0.001, 0.05, 3)
        pts = c[:, None] + rng.uniform(-1, 1, (3, 400)) * h[:, None]
        ant = rng.uniform(-0.07, 0.07, (3, 64))
        ant[2] = rng.uniform(-0.01, 0.01, 64)
        lo, hi = pts.min(1), pts.max(1)
        near = np.sqrt((np.maximum(np.maximum(lo[:, None] - ant, ant - hi[:, None]), 0.0) ** 2).sum(0)).min()
        far = np.sqrt((np.maximum(np.abs(ant - lo[:, None]), np.abs(hi[:, None] - ant)) ** 2).sum(0)).max()
        r = np.sqrt(((pts[:, :, None] - ant[:, None, :]) ** 2).sum(0))
        assert near <= r.min() + 1e-15 and r.max() <= far + 1e-15
        # tight for the box: the box's own corners reach the bounds
        corners = np.stack(np.meshgrid(*zip(lo, hi), indexing="ij"), 0).reshape(3, -1)
        rc = np.sqrt(((corners[:, :, None] - ant[:, None, :]) ** 2).sum(0))
        assert abs(rc.max() - far) < 1e-12
