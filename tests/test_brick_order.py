"""Host checks of the brick numbering the Chebyshev calls order points by
(tests/brick_order.py): a 3-D Hilbert curve over 8 x 8 x 8 bricks visits
every brick once and steps only between face neighbours, so consecutive
records stay spatially compact across brick boundaries."""
import numpy as np

from brick_order import brick_codes, brick_order, hilbert_brick


def test_hilbert_bricks_bijective_and_face_adjacent():
    cells = {}
    for x in range(8):
        for y in range(8):
            for z in range(8):
                cells[hilbert_brick(x, y, z)] = (x, y, z)
    assert sorted(cells) == list(range(512))
    steps = [np.abs(np.subtract(cells[h + 1], cells[h])).sum() for h in range(511)]
    assert all(s == 1 for s in steps)
    assert cells[0] == (0, 0, 0)


def test_hilbert_two_bit_curve_is_the_order_2_curve():
    """With one bit per axis the curve is the 8-corner Gray-code tour of the
    unit cube: consecutive corners differ in one coordinate."""
    corners = {hilbert_brick(x, y, z, bits=1): (x, y, z) for x in (0, 1) for y in (0, 1) for z in (0, 1)}
    assert sorted(corners) == list(range(8))
    assert all(np.abs(np.subtract(corners[h + 1], corners[h])).sum() == 1 for h in range(7))


def test_brick_order_runs_are_compact():
    """Uniform points of a cube, runs of n/512 consecutive records (about one
    brick's count, so most runs straddle two bricks): every run covers at
    most three consecutive bricks, hence a face-connected path of cells whose
    extent is at most one brick along its shortest axis, two along the next
    and three along the longest."""
    rng = np.random.default_rng(0)
    n = 512 * 64
    xyz = rng.uniform(0.0, 1.0, (3, n)).astype(np.float32)
    o = brick_order(xyz)
    rec, codes = xyz[:, o], brick_codes(xyz)[o]
    assert np.all(np.diff(codes) >= 0)
    for j in range(0, n, 64):
        assert codes[j + 63] - codes[j] <= 2
        ext = np.sort(rec[:, j:j + 64].max(1) - rec[:, j:j + 64].min(1))
        assert ext[0] <= 1.0 / 8 + 1e-6 and ext[1] <= 2.0 / 8 + 1e-6 and ext[2] <= 3.0 / 8 + 1e-6
