"""The record order of the Chebyshev phasor calls, stated on the host.

The points' bounding box is cut into 8 x 8 x 8 bricks (FP32 cell index per
axis) and the bricks are numbered along a 3-D Hilbert curve: J. Skilling,
"Programming the Hilbert curve", AIP Conf. Proc. 707 (2004), transpose form
(undo the excess work of the inverse transform plane by plane, Gray-encode,
read the index bits out plane-major). Records are the points stably sorted by
brick number.
"""
import numpy as np


def hilbert_brick(x: int, y: int, z: int, bits: int = 3) -> int:
    """Hilbert index of cell (x, y, z), `bits` bits per axis."""
    X = [int(x), int(y), int(z)]
    Q = 1 << (bits - 1)
    while Q > 1:
        P = Q - 1
        for i in range(3):
            if X[i] & Q:
                X[0] ^= P
            else:
                t = (X[0] ^ X[i]) & P
                X[0] ^= t
                X[i] ^= t
        Q >>= 1
    X[1] ^= X[0]
    X[2] ^= X[1]
    t, Q = 0, 1 << (bits - 1)
    while Q > 1:
        if X[2] & Q:
            t ^= Q - 1
        Q >>= 1
    X = [v ^ t for v in X]
    h = 0
    for j in range(bits - 1, -1, -1):
        for i in range(3):
            h = (h << 1) | ((X[i] >> j) & 1)
    return h


_TABLE = np.array([[[hilbert_brick(x, y, z) for z in range(8)] for y in range(8)] for x in range(8)],
                  dtype=np.int64)


def brick_codes(xyz) -> np.ndarray:
    """Brick number of every point ([3, n] coordinates, FP32 arithmetic)."""
    x = np.ascontiguousarray(xyz, dtype=np.float32)
    lo, hi = x.min(1), x.max(1)
    c = np.zeros((3, x.shape[1]), dtype=np.int64)
    for d in range(3):
        span = np.float32(hi[d] - lo[d])
        if span > 0:
            q = np.float32(8.0) / span
            c[d] = ((x[d] - lo[d]).astype(np.float32) * q).astype(np.float32).astype(np.int64)
        c[d] = np.clip(c[d], 0, 7)
    return _TABLE[c[0], c[1], c[2]]


def brick_order(xyz) -> np.ndarray:
    """Indices of the points in record order (stable sort by brick number)."""
    return np.argsort(brick_codes(xyz), kind="stable")
