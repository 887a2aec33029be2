"""Shared helpers of the GPU parity tests: which points sit away from the two
kinks of the render amplitude, where the FP32 kernel and the FP64 oracle may
take different (equally correct) one-sided derivatives.

- The directional factor D = max(2 c^2 - 1, 0) (App. A.3): its gradient in the
  normal jumps at 2 c^2 = 1.
- The lensless transmittance T' = clamp(t_eff - c_ant, 0, 1) (section 6,
  App. B.2): its slope in t_eff jumps at t_eff - c_ant = 0 and 1. The oracle
  decides the side on the exact FP64 difference, the kernel on the rounded
  FP32 one; near 1 the rounding can move a pair across the kink.
"""
import numpy as np


def away_from_directional_kink(xyz, grad, ant, margin):
    """Points none of whose (point, antenna) pairs has |2 c^2 - 1| < margin,
    c = cos of the angle between the point's gradient and the direction to
    the antenna (FP64); points with a zero gradient (isotropic) count as away."""
    x, gv, a = (np.asarray(v, np.float64) for v in (xyz, grad, ant))
    gn = np.linalg.norm(gv, axis=0)
    d = a[:, None, :] - x[:, :, None]                        # [3, n, n_ant]
    c = np.einsum("in,ina->na", gv, d) / (np.maximum(gn, 1e-300)[:, None] * np.linalg.norm(d, axis=0))
    near = (np.abs(2.0 * c * c - 1.0) < margin).any(axis=1)
    return ~near | (gn == 0.0)


def away_from_clamp_kink(t_eff, c_ant, margin=1e-6, chunk=4096):
    """Points none of whose (point, antenna) pairs has t_eff - c_ant (FP64)
    within `margin` of 0 or 1, the kinks of the lensless transmittance clamp
    (FP32 rounding of values below 2 is ~1.2e-7)."""
    t = np.asarray(t_eff, np.float64)
    c = np.asarray(c_ant, np.float64)
    away = np.ones(t.shape[0], dtype=bool)
    for j0 in range(0, t.shape[0], chunk):
        v = t[j0:j0 + chunk, None] - c[None, :]
        near = ((np.abs(v) < margin) | (np.abs(v - 1.0) < margin)).any(axis=1)
        away[j0:j0 + chunk] = ~near
    return away
