"""Learned proposal sampler on the GPU vs the FP64 oracle: network logits and
q, bit-exact inverse-CDF sampling from the kernel's own FP32 q, and the
training signal (weight histogram, KL loss, network and feature gradients)."""
import numpy as np
import pytest
import torch

import geraf_inputs as gi

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, np.float64); b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2605_29097_gb300 import _build
    _build.build()
    import paper_2605_29097_gb300 as G
    return G


def _prop(G, gshape=(8, 8, 16), F=8, width=64, n_hidden=3, depth=16, seed=0):
    G0, G1, G2 = gshape
    rng = np.random.default_rng(seed)
    feats = (rng.standard_normal((G2, G1, G0, F)) * 0.5).astype(np.float16)
    shapes = [(width, F)] + [(width, width)] * (n_hidden - 1) + [(1, width)]
    parts = []
    for o, i in shapes:
        parts += [rng.uniform(-1 / np.sqrt(i), 1 / np.sqrt(i), o * i), rng.uniform(-0.2, 0.2, o)]
    params = np.concatenate(parts).astype(np.float32)
    prop = G.Proposal(torch.as_tensor(feats, device="cuda"), torch.as_tensor(params, device="cuda"), width=width,
                      n_hidden=n_hidden, beta=10.0, eps=0.02, depth=depth)
    return prop, feats, params


def test_density_matches_oracle(G, oracle):
    prop, feats, params = _prop(G)
    logits, q, _ = G.geraf_proposal_density(prop)
    ol, _ = oracle.proposal_logits(feats.reshape(-1, 8), params, 64, 3, 10.0)
    assert rel(logits.cpu().numpy(), ol) < 1e-5
    oq = oracle.proposal_q(logits.cpu().numpy(), prop.gshape, 0.02)
    assert rel(q.cpu().numpy(), oq.reshape(-1)) < 1e-6


@pytest.mark.parametrize("n,depth", [((32, 24, 40), 16), ((8, 8, 16), 5)])
def test_sampling_bit_exact(G, oracle, n, depth):
    gshape = (8, 8, 16) if n[0] % 8 == 0 and n[1] % 8 == 0 else (4, 4, 16)
    prop, _, _ = _prop(G, gshape=gshape, depth=depth)
    logits, q, _ = G.geraf_proposal_density(prop)
    g = gi.cube_grid((0.0, 0.0, 0.15), 0.1, n)
    grid = G.make_grid(g.lo, g.pitch, g.n, g.aperture_z)
    xyz, apr, idx = G.geraf_sample_proposal(grid, prop, q, seed=77, step=5)
    q_np = q.cpu().numpy().reshape(gshape[2], gshape[1], gshape[0])
    oxyz, oapr, oidx = oracle.proposal_sample(g, gshape, q_np, depth, seed=77, step=5)
    np.testing.assert_array_equal(xyz.cpu().numpy().view(np.uint32), oxyz.view(np.uint32))
    np.testing.assert_array_equal(apr.cpu().numpy().view(np.uint32), oapr.view(np.uint32))
    np.testing.assert_array_equal(idx.cpu().numpy(), oidx)


@pytest.mark.parametrize("use_idx", [True, False])
def test_training_signal_matches_oracle(G, oracle, use_idx):
    prop, feats, params = _prop(G)
    logits, q, saved = G.geraf_proposal_density(prop)
    g = gi.cube_grid((0.0, 0.0, 0.15), 0.1, (32, 32, 32))
    grid = G.make_grid(g.lo, g.pitch, g.n)
    rng = np.random.default_rng(4)
    if use_idx:
        xyz, apr, idx = G.geraf_sample_proposal(grid, prop, q, seed=3, step=0)
        n_z = prop.depth
        idx_np = idx.cpu().numpy()
    else:
        idx = None
        n_z = g.n[2]
        k = np.arange(n_z)[:, None]
        ray = np.arange(g.n_ray)[None, :]
        ix, iy = ray % 32, ray // 32
        idx_np = (((k * 16 // n_z) * 8 + iy * 8 // 32) * 8 + ix * 8 // 32).reshape(-1)
    n = g.n_ray * n_z
    alpha = (rng.uniform(0, 1, n) * (rng.uniform(0, 1, n) > 0.7)).astype(np.float32)
    T = rng.uniform(0, 1, n).astype(np.float32)
    cu = lambda x: torch.as_tensor(x, device="cuda")
    d_p, d_f, loss = G.geraf_sample_backward(prop, grid, n_z, cu(alpha), cu(T), idx, logits, saved)
    hist = oracle.proposal_targets(T.astype(np.float64) * alpha, idx_np, prop.n_cells)
    oL, od = oracle.proposal_loss(logits.cpu().numpy(), prop.gshape, 0.02, hist)
    np.testing.assert_allclose(float(loss), oL, rtol=1e-6)
    _, cache = oracle.proposal_logits(feats.reshape(-1, 8), params, 64, 3, 10.0)
    odp, odf = oracle.proposal_backward(feats.reshape(-1, 8), params, 64, 3, 10.0, cache, od)
    assert rel(d_p.cpu().numpy(), odp) < 1e-5
    assert rel(d_f.cpu().numpy().reshape(-1, 8), odf) < 1e-5


@pytest.mark.parametrize("m,r_max,dilate", [(5, 2, 0), (16, 16, 0), (1, 0, 0), (6, 3, 1), (9, 2, 2)])
def test_sample_cells_bit_exact(G, oracle, m, r_max, dilate):
    """Cell-subset sampling from the network's own FP32 q (with ties planted
    in q): points, ray starts, cell indices and keep flags bit-exact with the
    oracle, which takes the points from the dense stratified grid."""
    prop, _, _ = _prop(G, gshape=(8, 4, 16))
    g = gi.cube_grid((0.0, 0.0, 0.15), 0.08, (32, 24, 64))
    grid = G.make_grid(g.lo, g.pitch, g.n, g.aperture_z)
    _, q, _ = G.geraf_proposal_density(prop)
    qh = q.cpu().numpy().copy().reshape(16, 4 * 8)      # [gz][gy gx]
    qh[3, :] = qh[7, :]                                   # ties between cells 3 and 7 of every column
    qh = qh.ravel()
    q = torch.as_tensor(qh, device="cuda")
    xyz, apr, idx, keep, n_out = G.geraf_sample_cells(grid, prop, q, m, r_max, seed=5, step=3, dilate=dilate)
    G.geraf_poll_device_error()
    ox, oa, oi, ok, on = oracle.sample_cells(g, (8, 4, 16), qh, m, r_max, seed=5, step=3, dilate=dilate)
    assert n_out == on
    np.testing.assert_array_equal(xyz.cpu().numpy().view(np.uint32), ox.view(np.uint32))
    np.testing.assert_array_equal(apr.cpu().numpy().view(np.uint32), oa.view(np.uint32))
    np.testing.assert_array_equal(idx.cpu().numpy(), oi)
    np.testing.assert_array_equal(keep.cpu().numpy(), ok)


def test_blend_keep_and_backward(G, oracle):
    """geraf_blend with a keep mask (w = keep a alpha A'_tx) and its adjoint
    against the oracle at 1e-5 (the dL/df tolerance of the plain blend, 1e-4)."""
    rng = np.random.default_rng(12)
    n_ray, n_z = 301, 37
    sdf = np.cumsum(-rng.uniform(0.0, 0.002, (n_z, n_ray)), axis=0).astype(np.float32).ravel() + 0.02
    refl = rng.uniform(0.2, 1.0, n_ray * n_z).astype(np.float32)
    keep = (rng.uniform(0, 1, n_ray * n_z) < 0.7).astype(np.float32)
    apr = rng.uniform(-0.01, 0.03, n_ray).astype(np.float32)
    ant = rng.uniform(-0.01, 0.03, 17).astype(np.float32)
    s, atx = np.float32(500.0), np.float32(1.3)
    cu = lambda x: torch.as_tensor(x, device="cuda")
    al, T, w, te, ca = G.geraf_blend(cu(sdf), cu(refl), n_ray, n_z, cu(apr), cu(ant), float(s), float(atx), cu(keep))
    G.geraf_poll_device_error()
    oal, oT, ow, ote, oca = oracle.blend(sdf, refl, n_ray, n_z, apr, ant, s, atx, keep)
    assert rel(w.cpu().numpy(), ow) < 1e-5 and rel(T.cpu().numpy(), oT) < 1e-5
    assert np.all(w.cpu().numpy()[keep == 0] == 0.0)
    d_w = rng.standard_normal(n_ray * n_z).astype(np.float32)
    d_t = rng.standard_normal(n_ray * n_z).astype(np.float32)
    d_f, d_a, d_sc = G.geraf_blend_backward(cu(sdf), cu(refl), al, T, n_ray, n_z, float(s), float(atx), cu(d_w),
                                            cu(d_t), cu(keep))
    G.geraf_poll_device_error()
    od_f, od_a, od_s, od_atx = oracle.blend_backward(sdf, refl, n_ray, n_z, s, atx, d_w, d_t, keep)
    assert rel(d_f.cpu().numpy(), od_f) < 1e-4
    assert rel(d_a.cpu().numpy(), od_a) < 1e-5
    np.testing.assert_allclose(d_sc.cpu().numpy(), [od_s, od_atx], rtol=1e-4)
