"""geraf_render_noalloc: signal tracing that takes no workspace, for callers
that cannot allocate device memory (its scratch is a static device array of
the library). Called through the C ABI on two calls in a row and compared
with geraf_render; oversized inputs are refused with a status code. Kept in a
file of its own, collected last."""
import ctypes

import numpy as np
import pytest
import torch

import geraf_inputs as gi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2605_29097_gb300 import _build
    _build.build()
    import paper_2605_29097_gb300 as G
    return G


def _inputs(rng, n_pts, n_side, n_f):
    xyz = (np.array([0.0, 0.0, 0.15])[:, None] + rng.uniform(-0.05, 0.05, (3, n_pts))).astype(np.float32)
    grad = rng.standard_normal((3, n_pts)).astype(np.float32)
    w = rng.uniform(0, 1, n_pts).astype(np.float32)
    t_eff = rng.uniform(0.3, 2.0, n_pts).astype(np.float32)
    ant = gi.antenna_array(n_side, n_side, 0.002)
    c_ant = rng.uniform(0.2, 1.0, ant.shape[1]).astype(np.float32)
    cu = lambda x: torch.as_tensor(x, device="cuda")
    return [cu(v) for v in (xyz, grad, w, t_eff, ant, c_ant)], gi.band(77e9, 81e9, n_f)


def _noalloc(G, xyz, grad, w, t_eff, ant, c_ant, b):
    from paper_2605_29097_gb300 import _lib
    out = torch.empty(ant.shape[1], b.n_f, 2, dtype=torch.float32, device="cuda")
    band = _lib.GerafBand(b.f0, b.df, b.n_f)
    vp = lambda t: ctypes.c_void_p(t.data_ptr())
    st = _lib.lib().geraf_render_noalloc(vp(xyz), vp(grad), vp(w), vp(t_eff), xyz.shape[1], vp(ant), vp(c_ant),
                                         ant.shape[1], ctypes.byref(band), 1, vp(out),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, out


def _rel(a, b):
    return float(torch.linalg.norm((a - b).double()) / torch.linalg.norm(b.double()))


# (5003, 10, 96): 64 bins and more, where geraf_render runs its Chebyshev form
# and the no-allocation call still runs the per-bin recurrence;
# (600 001, 16, 512): 28.8 MB of packed points leave room for only 4 of the
# 1 MB split partials, so the call merges point tiles into fewer splits.
@pytest.mark.parametrize("n_pts,n_side,n_f", [(5003, 10, 45), (32769, 16, 32), (5003, 10, 96),
                                              (600001, 16, 512)])
def test_noalloc_matches_render_twice(G, n_pts, n_side, n_f):
    rng = np.random.default_rng(n_pts)
    args, b = _inputs(rng, n_pts, n_side, n_f)
    want = torch.view_as_real(G.geraf_render(*args, G.Band(b.f0, b.df, b.n_f)))
    for _ in range(2):
        st, got = _noalloc(G, *args, b)
        assert st == 0
        torch.cuda.synchronize()
        G.geraf_poll_device_error()
        assert _rel(got, want) < 1e-5


def test_noalloc_refuses_oversized_input(G):
    from paper_2605_29097_gb300 import _lib
    rng = np.random.default_rng(1)
    args, b = _inputs(rng, 1_000_000, 8, 32)        # 48 MB of packed points > 32 MiB
    st, _ = _noalloc(G, *args, b)
    assert st == 6
    assert b"static limit" in _lib.lib().geraf_last_error_string()
