"""Pins for the oracle's lensless sampling and its counter-based generator."""
import os

import numpy as np
from scipy import stats

import geraf_inputs as gi

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_splitmix():
    for line in open(os.path.join(GOLDEN, "splitmix64.txt")):
        if line.startswith("seed"):
            parts = line.split()
            return int(parts[1]), int(parts[3], 16)
    raise AssertionError


def test_splitmix64_published_first_output(oracle):
    seed, out0 = _golden_splitmix()
    assert int(oracle.splitmix64(seed, 0)) == out0


def test_uniform01_is_uniform_and_streams_independent(oracle):
    idx = np.arange(200_000)
    u0 = oracle.uniform01(7, 3, 0, idx)
    u1 = oracle.uniform01(7, 3, 1, idx)
    u2 = oracle.uniform01(7, 4, 0, idx)
    for u in (u0, u1, u2):
        assert u.min() >= 0.0 and u.max() < 1.0
        assert stats.kstest(u, "uniform").pvalue > 1e-4
    assert abs(np.corrcoef(u0, u1)[0, 1]) < 0.01
    assert abs(np.corrcoef(u0, u2)[0, 1]) < 0.01
    # exact multiples of 2^-53
    assert np.all(u0 * 2.0 ** 53 == np.floor(u0 * 2.0 ** 53))


def test_uniform_grid_is_cell_centres_depth_major(oracle):
    g = gi.cube_grid((0.0, 0.0, 0.15), 0.10, (8, 6, 5))
    xyz, apr = oracle.sample(g, gi.SAMPLE_UNIFORM)
    nx, ny, nz = g.n
    for d in range(3):
        edges = np.float64(g.lo[d]) + np.arange(g.n[d] + 1) * np.float64(g.pitch[d])
        centres = 0.5 * (edges[:-1] + edges[1:])
        coord = xyz[d].reshape(nz, ny, nx)
        idx = {0: np.arange(nx)[None, None, :], 1: np.arange(ny)[None, :, None],
               2: np.arange(nz)[:, None, None]}[d]
        want = np.broadcast_to(centres[idx], coord.shape)
        np.testing.assert_allclose(coord, want, rtol=0, atol=2e-8)
    np.testing.assert_array_equal(apr[0], xyz[0][: nx * ny])
    np.testing.assert_array_equal(apr[1], xyz[1][: nx * ny])
    assert np.all(apr[2] == np.float32(g.aperture_z))


def test_stratified_inside_cells_and_columns_straight(oracle):
    g = gi.cube_grid((0.0, 0.0, 0.15), 0.10, (16, 8, 12))
    xyz, apr = oracle.sample(g, gi.SAMPLE_STRATIFIED, seed=11, step=2)
    nx, ny, nz = g.n
    P = xyz.reshape(3, nz, ny, nx).astype(np.float64)
    cell = [np.arange(nx)[None, None, :], np.arange(ny)[None, :, None], np.arange(nz)[:, None, None]]
    for d in range(3):
        lo = np.float64(g.lo[d]) + cell[d] * np.float64(g.pitch[d])
        hi = lo + np.float64(g.pitch[d])
        eps = 1e-7
        assert np.all(P[d] >= lo - eps) and np.all(P[d] <= hi + eps)
    # primary rays are parallel to +z: x, y constant along depth
    assert np.all(P[0] == P[0][:1]) and np.all(P[1] == P[1][:1])
    # jitter differs between steps, repeats for the same (seed, step)
    xyz2, _ = oracle.sample(g, gi.SAMPLE_STRATIFIED, seed=11, step=3)
    xyz3, _ = oracle.sample(g, gi.SAMPLE_STRATIFIED, seed=11, step=2)
    assert np.any(xyz2 != xyz)
    np.testing.assert_array_equal(xyz3, xyz)
    # within-cell offsets are uniform
    off = (P[2] - (np.float64(g.lo[2]) + cell[2] * np.float64(g.pitch[2]))) / np.float64(g.pitch[2])
    assert stats.kstest(off.reshape(-1), "uniform").pvalue > 1e-4
