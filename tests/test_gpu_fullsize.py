"""The four phasor sums at the full size of the 128x128-antenna, 256-bin,
256^3-sample workload, in the launch configuration the benchmark times
(Chebyshev form: 512 splits of one brick x 128 antenna blocks to bins, 512
point groups x 128 antenna blocks to points, the 24-order kernel instance),
checked against the FP64 oracle on sampled outputs the oracle computes one by
one:

- render: the signal of three antennas (two corners and the centre of the
  array) over all 256 bins, each a sum over all 2^24 points (section 5.1,
  Eq. ref_sim);
- render adjoint: w, t_eff and gradient adjoints of 48 random points, each a
  sum over all 16384 antennas and 256 bins (App. A.5);
- filter: M and P of 48 random voxels of the 64^3 heatmap grid (section 3,
  Eq. mf-sm);
- filter adjoint: the bins of two antennas, each a sum over all 262144 voxels.

Inputs are seeded and host-made: the stratified samples from the oracle's
sampler, random normals, weights in [0, 1), t_eff in [0.3, 2], c_ant in
[0.2, 1], random complex signals and filter outputs. Tolerance 1e-5 relative
L2 (3e-5 for the gradient adjoint), with the points near the clamp's and the
directional factor's kinks excluded (within 1e-6 and 1e-5).
"""
import numpy as np
import pytest
import torch

import geraf_inputs as gi
from parity_helpers import away_from_clamp_kink, away_from_directional_kink

pytestmark = pytest.mark.gpu

TOL = 1e-5


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.complex128 if np.iscomplexobj(a) else np.float64)
    b = np.asarray(b, dtype=a.dtype)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def cu(x):
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float32), device="cuda")


def host(t):
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2605_29097_gb300 import _build
    _build.build()
    import paper_2605_29097_gb300 as G
    return G


@pytest.fixture(scope="module")
def scene(oracle):
    wl = gi.workload("c3")
    assert wl.array_n == 128 and wl.n_f == 256 and wl.grid.n == (256, 256, 256)
    xyz, _ = oracle.sample(wl.grid, gi.SAMPLE_STRATIFIED, seed=7, step=0)
    vox, _ = oracle.sample(wl.heat, gi.SAMPLE_UNIFORM)
    n = xyz.shape[1]
    rng = np.random.default_rng(71)
    grad = rng.standard_normal((3, n)).astype(np.float32)
    grad[:, ::17] = 0.0                                  # some isotropic points
    w = rng.uniform(0.0, 1.0, n).astype(np.float32)
    t_eff = rng.uniform(0.3, 2.0, n).astype(np.float32)
    ant = gi.antenna_array(wl.array_n, wl.array_n, wl.array_pitch)
    c_ant = rng.uniform(0.2, 1.0, ant.shape[1]).astype(np.float32)
    b = gi.band(77e9, 81e9, wl.n_f)
    return dict(xyz=xyz.astype(np.float32), vox=vox.astype(np.float32), grad=grad, w=w, t_eff=t_eff,
                ant=ant, c_ant=c_ant, b=b, rng=rng)


def test_fullsize_launch_configuration(G, scene):
    """The plan the benchmark's calls run at this size: the Chebyshev form with
    the 24-order instance, parts of at most 12 orders, 8 to 9 orders per pair."""
    sc = scene
    band = G.Band(sc["b"].f0, sc["b"].df, sc["b"].n_f)
    for to_points in (False, True):
        k0, km, inst, mean = G.geraf_chebyshev_work(cu(sc["xyz"]), cu(sc["ant"]), band, to_points)
        assert k0 > 0 and inst == 24 and km <= 12, (k0, km, inst, mean)
        assert 8.0 <= mean <= 10.0, mean


def test_fullsize_render_and_adjoint(G, oracle, scene):
    sc = scene
    xyz, grad, w, t_eff, ant, c_ant, b = (sc[k] for k in ("xyz", "grad", "w", "t_eff", "ant", "c_ant", "b"))
    band = G.Band(b.f0, b.df, b.n_f)
    s = G.geraf_render(cu(xyz), cu(grad), cu(w), cu(t_eff), cu(ant), cu(c_ant), band, True)
    G.geraf_poll_device_error()
    aidx = np.array([0, 128 * 64 + 64, ant.shape[1] - 1])
    want = oracle.render(xyz, grad, w, t_eff, ant[:, aidx], c_ant[aidx], b)
    err = rel_l2(host(s)[aidx], want)
    print("render, 3 antennas x 256 bins over 2^24 points: rel L2", err)
    assert err < TOL

    rng = sc["rng"]
    g_s = gi.complex_normal(rng, (ant.shape[1], b.n_f)).astype(np.complex64)
    d_w, d_t, d_g = G.geraf_render_backward(cu(xyz), cu(grad), cu(w), cu(t_eff), cu(ant), cu(c_ant), band,
                                            torch.as_tensor(g_s, device="cuda"))
    G.geraf_poll_device_error()
    pidx = np.sort(rng.choice(xyz.shape[1], 48, replace=False))
    ow, ot, og = oracle.render_backward(xyz[:, pidx], grad[:, pidx], w[pidx], t_eff[pidx], ant, c_ant, b, g_s)
    kt = away_from_clamp_kink(t_eff[pidx], c_ant)
    # with 16384 antennas most points have some pair within 1e-4 of the
    # directional factor's kink; a pair can take the other side in FP32 than in
    # FP64 only within its rounding (~1e-6), so the margin here is 1e-5
    away = away_from_directional_kink(xyz[:, pidx], grad[:, pidx], ant, 1e-5)
    e_w = rel_l2(host(d_w)[pidx], ow)
    e_t = rel_l2(host(d_t)[pidx][kt], ot[kt])
    e_g = rel_l2(host(d_g)[:, pidx][:, away], og[:, away])
    print("render adjoint, 48 points x 16384 antennas x 256 bins: rel L2 w", e_w, "t_eff", e_t, "G", e_g,
          "(", int(kt.sum()), "and", int(away.sum()), "of 48 points away from the kinks)")
    assert kt.sum() >= 40 and away.sum() >= 20
    assert e_w < TOL and e_t < TOL and e_g < 3 * TOL


def test_fullsize_filter_and_adjoint(G, oracle, scene):
    sc = scene
    vox, ant, b, rng = sc["vox"], sc["ant"], sc["b"], sc["rng"]
    band = G.Band(b.f0, b.df, b.n_f)
    n_vox = vox.shape[1]
    s_in = gi.complex_normal(rng, (ant.shape[1], b.n_f)).astype(np.complex64)
    P, M, _, _ = G.geraf_filter(torch.as_tensor(s_in, device="cuda"), cu(ant), band, cu(vox))
    G.geraf_poll_device_error()
    vidx = np.sort(rng.choice(n_vox, 48, replace=False))
    oM, oP = oracle.filter_forward(s_in, ant, vox[:, vidx], b)
    e_m, e_p = rel_l2(host(M)[vidx], oM), rel_l2(host(P)[vidx], oP)
    print("filter, 48 voxels x 16384 antennas x 256 bins: rel L2 M", e_m, "P", e_p)
    assert e_m < TOL and e_p < TOL

    M_in = gi.complex_normal(rng, n_vox).astype(np.complex64)
    d_P = rng.standard_normal(n_vox).astype(np.float32)
    gb = G.geraf_filter_backward(cu(ant), band, cu(vox), torch.as_tensor(M_in, device="cuda"), cu(d_P))
    G.geraf_poll_device_error()
    aidx = np.array([127, 128 * 100 + 30])
    og = oracle.filter_backward(M_in, d_P, ant[:, aidx], vox, b)
    e_g = rel_l2(host(gb)[aidx], og)
    print("filter adjoint, 2 antennas x 256 bins over 262144 voxels: rel L2", e_g)
    assert e_g < TOL
