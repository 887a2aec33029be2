"""Pins for the oracle's fields: analytic SDFs against closed forms and finite
differences; the MLP (value, gradient tangents and hand-written adjoint)
against torch FP64 autograd on the same weights."""
import numpy as np
import pytest
import torch

import geraf_inputs as gi


def _fd_grad(fn, x, h=1e-6):
    g = np.zeros_like(x)
    for d in range(3):
        e = np.zeros_like(x); e[d] = h
        g[d] = (fn(x + e) - fn(x - e)) / (2 * h)
    return g


def test_sphere_closed_form(oracle):
    sc = gi.Scene([gi.Prim(gi.PRIM_SPHERE, 0.7, (0.01, -0.02, 0.15), (0.03, 0, 0))])
    x = np.array([[0.01, 0.01, 0.01 + 0.05], [-0.02, -0.02, -0.02], [0.15, 0.15 + 0.02, 0.15]])
    f, G, a = oracle.analytic_fields(sc, x)
    np.testing.assert_allclose(f, [-0.03, 0.02 - 0.03, 0.05 - 0.03], atol=1e-15)
    np.testing.assert_allclose(G[:, 1], [0, 0, 1], atol=1e-15)
    np.testing.assert_allclose(G[:, 2], [1, 0, 0], atol=1e-15)
    assert np.all(a == 0.7)


@pytest.mark.parametrize("kind,p", [(gi.PRIM_SPHERE, (0.03, 0, 0)), (gi.PRIM_BOX, (0.02, 0.01, 0.015)),
                                    (gi.PRIM_ELLIPSOID, (0.04, 0.02, 0.03)),
                                    (gi.PRIM_HALFSPACE, (0.0, 0.6, -0.8))])
def test_gradient_matches_finite_differences(oracle, kind, p):
    sc = gi.Scene([gi.Prim(kind, 1.0, (0.005, -0.004, 0.15), p)])
    rng = np.random.default_rng(3)
    x = np.array([0.0, 0.0, 0.15])[:, None] + rng.uniform(-0.06, 0.06, size=(3, 400))
    _, G, _ = oracle.analytic_fields(sc, x)
    Gfd = _fd_grad(lambda y: oracle.analytic_fields(sc, y)[0], x)
    # box SDF has gradient kinks on the medial axis: compare where smooth
    ok = np.abs(Gfd - G).max(0) < 1e-4
    assert ok.mean() > 0.97
    if kind != gi.PRIM_ELLIPSOID:
        np.testing.assert_allclose(np.linalg.norm(G, axis=0), 1.0, atol=1e-12)


def test_box_and_ellipsoid_distances(oracle):
    box = gi.Scene([gi.Prim(gi.PRIM_BOX, 1.0, (0, 0, 0.1), (0.02, 0.01, 0.03))])
    x = np.array([[0.05, 0.0, 0.0, 0.03], [0.0, 0.0, 0.0, 0.02], [0.1, 0.1, 0.2, 0.1 + 0.04]])
    f, _, _ = oracle.analytic_fields(box, x)
    np.testing.assert_allclose(f, [0.03, -0.01, 0.07, np.sqrt(0.01**2 + 0.01**2 + 0.01**2)], atol=1e-15)
    ell = gi.Scene([gi.Prim(gi.PRIM_ELLIPSOID, 1.0, (0, 0, 0.1), (0.04, 0.02, 0.03))])
    # exact along the smallest semi-axis
    x = np.array([[0.0, 0.0], [0.05, 0.01], [0.1, 0.1]])
    f, _, _ = oracle.analytic_fields(ell, x)
    np.testing.assert_allclose(f, [0.03, -0.01], atol=1e-15)


def test_union_takes_nearest_primitive(oracle):
    sc = gi.Scene([gi.Prim(gi.PRIM_SPHERE, 0.2, (0, 0, 0.1), (0.01, 0, 0)),
                   gi.Prim(gi.PRIM_SPHERE, 0.9, (0, 0, 0.2), (0.01, 0, 0))])
    x = np.array([[0.0, 0.0], [0.0, 0.0], [0.12, 0.17]])
    f, G, a = oracle.analytic_fields(sc, x)
    np.testing.assert_allclose(f, [0.01, 0.02], atol=1e-15)
    np.testing.assert_allclose(a, [0.2, 0.9])
    np.testing.assert_allclose(G[2], [1.0, -1.0])


def _torch_mlp(spec, params, xyz):
    """Independent autograd reference of the same network."""
    shapes = spec.shapes()
    p = torch.tensor(params.astype(np.float64), requires_grad=True)
    x = torch.tensor(xyz.T.astype(np.float64), requires_grad=True)
    # the network description carries center and half as FP32 values
    c = torch.tensor(np.asarray(spec.center, np.float32).astype(np.float64))
    xt = (x - c) / float(np.float32(spec.half))
    feats = []
    for k in range(spec.n_levels):
        feats.append(torch.sin((2.0 ** k) * np.pi * xt))
        feats.append(torch.cos((2.0 ** k) * np.pi * xt))
    z = torch.cat(feats, dim=1)
    off = 0
    for li, (o, i) in enumerate(shapes):
        W = p[off:off + o * i].view(o, i); off += o * i
        b = p[off:off + o]; off += o
        z = z @ W.T + b
        if li < len(shapes) - 1:
            z = torch.nn.functional.softplus(z, beta=spec.beta, threshold=1e6)
    f, a = z[:, 0], torch.sigmoid(z[:, 1])
    G = torch.autograd.grad(f.sum(), x, create_graph=True)[0]
    return p, f, G, a


def test_mlp_matches_torch_autograd(oracle):
    spec = gi.MLPSpec(n_levels=3, width=16, n_hidden=3, beta=20.0)
    params = gi.mlp_init(spec, seed=5)
    rng = np.random.default_rng(1)
    xyz = (np.array(spec.center)[:, None] + rng.uniform(-0.05, 0.05, (3, 37))).astype(np.float32)
    f, G, a, cache = oracle.mlp_forward(spec, params, xyz)
    p, tf, tG, ta = _torch_mlp(spec, params, xyz)
    np.testing.assert_allclose(f, tf.detach().numpy(), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(a, ta.detach().numpy(), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(G, tG.detach().numpy().T, rtol=1e-10, atol=1e-11)
    d_f, d_G, d_a = rng.standard_normal(37), rng.standard_normal((3, 37)), rng.standard_normal(37)
    gp = oracle.mlp_backward(spec, params, cache, d_f, d_G, d_a)
    L = (tf * torch.tensor(d_f)).sum() + (tG * torch.tensor(d_G.T)).sum() + (ta * torch.tensor(d_a)).sum()
    tgp = torch.autograd.grad(L, p)[0].numpy()
    np.testing.assert_allclose(gp, tgp, rtol=1e-9, atol=1e-10 * np.abs(tgp).max())


def _torch_bf16_streams(spec, params, xyz):
    """Independent reference of the BF16 network (reading: hidden weights and
    every hidden layer's inputs, value and tangents, rounded to bfloat16; head
    weights FP32): value and the three x-tangents as explicit streams, the
    tangents of the encoding by forward-mode AD, rounding by torch's own
    float32 -> bfloat16 cast with a straight-through gradient, parameter
    gradient by reverse-mode autograd."""
    from torch.func import jvp
    shapes = spec.shapes()
    p = torch.tensor(params.astype(np.float64), requires_grad=True)
    x = torch.tensor(xyz.T.astype(np.float64))
    c = torch.tensor(np.asarray(spec.center, np.float32).astype(np.float64))
    half = float(np.float32(spec.half))

    def pe(xx):
        xt = (xx - c) / half
        feats = []
        for k in range(spec.n_levels):
            feats.append(torch.sin((2.0 ** k) * np.pi * xt))
            feats.append(torch.cos((2.0 ** k) * np.pi * xt))
        return torch.cat(feats, dim=1)

    def rnd(t):
        return t + (t.to(torch.float32).to(torch.bfloat16).to(torch.float64) - t).detach()

    z = pe(x)
    dz = [jvp(pe, (x,), (torch.nn.functional.one_hot(torch.full((x.shape[0],), d), 3).double(),))[1]
          for d in range(3)]
    off = 0
    for li, (o, i) in enumerate(shapes):
        W = p[off:off + o * i].view(o, i); off += o * i
        b = p[off:off + o]; off += o
        if li < len(shapes) - 1:
            Wr, zr, dzr = rnd(W), rnd(z), [rnd(t) for t in dz]
            h = zr @ Wr.T + b
            dh = [t @ Wr.T for t in dzr]
            s = torch.sigmoid(spec.beta * h)
            z = torch.nn.functional.softplus(h, beta=spec.beta, threshold=1e6)
            dz = [s * t for t in dh]
        else:
            zr, dzr = rnd(z), [rnd(t) for t in dz]
            out = zr @ W.T + b
            f, a = out[:, 0], torch.sigmoid(out[:, 1])
            G = torch.stack([t @ W[0] for t in dzr], 1)
    return p, f, G, a


def test_mlp_bf16_network_and_straight_through_adjoint_match_torch(oracle):
    spec = gi.MLPSpec(n_levels=3, width=16, n_hidden=3, beta=20.0)
    params = gi.mlp_init(spec, seed=6)
    rng = np.random.default_rng(2)
    xyz = (np.array(spec.center)[:, None] + rng.uniform(-0.05, 0.05, (3, 41))).astype(np.float32)
    f, G, a, cache = oracle.mlp_forward(spec, params, xyz, precision="bf16")
    p, tf, tG, ta = _torch_bf16_streams(spec, params, xyz)
    np.testing.assert_allclose(f, tf.detach().numpy(), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(a, ta.detach().numpy(), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(G, tG.detach().numpy().T, rtol=1e-10, atol=1e-11)
    # the BF16 network differs from the FP32 one by the roundings (a dropped rounding would not)
    f32, _, _, _ = oracle.mlp_forward(spec, params, xyz)
    assert np.abs(f - f32).max() > 1e-6
    d_f, d_G, d_a = rng.standard_normal(41), rng.standard_normal((3, 41)), rng.standard_normal(41)
    gp = oracle.mlp_backward(spec, params, cache, d_f, d_G, d_a)
    L = (tf * torch.tensor(d_f)).sum() + (tG * torch.tensor(d_G.T)).sum() + (ta * torch.tensor(d_a)).sum()
    tgp = torch.autograd.grad(L, p)[0].numpy()
    np.testing.assert_allclose(gp, tgp, rtol=1e-9, atol=1e-10 * np.abs(tgp).max())


def _torch_nets(nets, params, xyz):
    """Independent autograd reference of the paper's two networks: the SDF
    network's f and its x-gradient (reverse-mode through the encoding), the
    reflectivity network's sigmoid output, from the same packed parameters."""
    p = torch.tensor(params.astype(np.float64), requires_grad=True)
    x = torch.tensor(xyz.T.astype(np.float64), requires_grad=True)

    def net(spec, q):
        c = torch.tensor(np.asarray(spec.center, np.float32).astype(np.float64))
        xt = (x - c) / float(np.float32(spec.half))
        z = torch.cat([f((2.0 ** k) * np.pi * xt) for k in range(spec.n_levels) for f in (torch.sin, torch.cos)], 1)
        off = 0
        shapes = spec.shapes()
        for li, (o, i) in enumerate(shapes):
            W = q[off:off + o * i].view(o, i); off += o * i
            b = q[off:off + o]; off += o
            z = z @ W.T + b
            if li < len(shapes) - 1:
                z = torch.nn.functional.softplus(z, beta=spec.beta, threshold=1e6)
        return z[:, 0]

    ns = nets.sdf.n_params
    f = net(nets.sdf, p[:ns])
    a = torch.sigmoid(net(nets.refl, p[ns:]))
    G = torch.autograd.grad(f.sum(), x, create_graph=True)[0]
    return p, f, G, a


@pytest.mark.parametrize("paper_size", [False, True])
def test_two_networks_match_torch_autograd(oracle, paper_size):
    """The paper's separate SDF and reflectivity networks (App. C): values,
    SDF gradient and the adjoint of all packed parameters; the small case
    checks every code path quickly, the paper-size case (8 x 256 and 4 x 256,
    10 octaves) the shapes the GPU runs."""
    if paper_size:
        nets, n = gi.paper_nets(), 5
    else:
        nets = gi.FieldNets(gi.MLPSpec(4, 24, 3, 30.0, (0.0, 0.0, 0.15), 0.05, 1),
                            gi.MLPSpec(4, 16, 2, 30.0, (0.0, 0.0, 0.15), 0.05, 1))
        n = 29
    params = gi.nets_init(nets, seed=7, sdf_bias=0.01)
    assert params.size == nets.n_params
    rng = np.random.default_rng(4)
    xyz = (np.array([0.0, 0.0, 0.15])[:, None] + rng.uniform(-0.05, 0.05, (3, n))).astype(np.float32)
    f, G, a, cache = oracle.nets_forward(nets, params, xyz)
    p, tf, tG, ta = _torch_nets(nets, params, xyz)
    np.testing.assert_allclose(f, tf.detach().numpy(), rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(a, ta.detach().numpy(), rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(G, tG.detach().numpy().T, rtol=1e-9, atol=1e-10 * np.abs(G).max())
    d_f, d_G, d_a = rng.standard_normal(n), rng.standard_normal((3, n)), rng.standard_normal(n)
    gp = oracle.nets_backward(nets, params, cache, d_f, d_G, d_a)
    L = (tf * torch.tensor(d_f)).sum() + (tG * torch.tensor(d_G.T)).sum() + (ta * torch.tensor(d_a)).sum()
    tgp = torch.autograd.grad(L, p)[0].numpy()
    np.testing.assert_allclose(gp, tgp, rtol=1e-8, atol=1e-10 * np.abs(tgp).max())
    # the reflectivity network's block gets its own gradient (a dropped d_a would zero it)
    assert np.abs(gp[nets.sdf.n_params:]).max() > 0


def _torch_bf16_net(spec, q, x):
    """One network of the BF16 reading as explicit value and tangent streams
    (hidden weights and every hidden layer's inputs rounded to bfloat16 by
    torch's own cast, straight-through gradient; head FP32): (out, tangents)
    of its single output."""
    from torch.func import jvp
    c = torch.tensor(np.asarray(spec.center, np.float32).astype(np.float64))
    half = float(np.float32(spec.half))

    def pe(xx):
        xt = (xx - c) / half
        return torch.cat([f((2.0 ** k) * np.pi * xt) for k in range(spec.n_levels) for f in (torch.sin, torch.cos)], 1)

    def rnd(t):
        return t + (t.to(torch.float32).to(torch.bfloat16).to(torch.float64) - t).detach()

    z = pe(x)
    dz = [jvp(pe, (x,), (torch.nn.functional.one_hot(torch.full((x.shape[0],), d), 3).double(),))[1]
          for d in range(3)]
    off = 0
    shapes = spec.shapes()
    for li, (o, i) in enumerate(shapes):
        W = q[off:off + o * i].view(o, i); off += o * i
        b = q[off:off + o]; off += o
        zr, dzr = rnd(z), [rnd(t) for t in dz]
        if li < len(shapes) - 1:
            Wr = rnd(W)
            h = zr @ Wr.T + b
            dh = [t @ Wr.T for t in dzr]
            s = torch.sigmoid(spec.beta * h)
            z = torch.nn.functional.softplus(h, beta=spec.beta, threshold=1e6)
            dz = [s * t for t in dh]
        else:
            return (zr @ W.T + b)[:, 0], torch.stack([t @ W[0] for t in dzr], 1)


def test_two_networks_bf16_match_torch(oracle):
    """The BF16 reading applied to the paper's two networks (a small shape of
    the same structure): values, SDF gradient and the straight-through adjoint
    of all packed parameters against an explicit torch construction."""
    nets = gi.FieldNets(gi.MLPSpec(4, 24, 3, 30.0, (0.0, 0.0, 0.15), 0.05, 1),
                        gi.MLPSpec(4, 16, 2, 30.0, (0.0, 0.0, 0.15), 0.05, 1))
    n = 31
    params = gi.nets_init(nets, seed=8, sdf_bias=0.01)
    rng = np.random.default_rng(6)
    xyz = (np.array([0.0, 0.0, 0.15])[:, None] + rng.uniform(-0.05, 0.05, (3, n))).astype(np.float32)
    f, G, a, cache = oracle.nets_forward(nets, params, xyz, precision="bf16")
    p = torch.tensor(params.astype(np.float64), requires_grad=True)
    x = torch.tensor(xyz.T.astype(np.float64))
    ns = nets.sdf.n_params
    tf, tG = _torch_bf16_net(nets.sdf, p[:ns], x)
    tl, _ = _torch_bf16_net(nets.refl, p[ns:], x)
    ta = torch.sigmoid(tl)
    np.testing.assert_allclose(f, tf.detach().numpy(), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(a, ta.detach().numpy(), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(G, tG.detach().numpy().T, rtol=1e-10, atol=1e-11 * np.abs(G).max())
    f32, _, _, _ = oracle.nets_forward(nets, params, xyz)
    assert np.abs(f - f32).max() > 1e-6                  # the roundings are applied
    d_f, d_G, d_a = rng.standard_normal(n), rng.standard_normal((3, n)), rng.standard_normal(n)
    gp = oracle.nets_backward(nets, params, cache, d_f, d_G, d_a)
    L = (tf * torch.tensor(d_f)).sum() + (tG * torch.tensor(d_G.T)).sum() + (ta * torch.tensor(d_a)).sum()
    tgp = torch.autograd.grad(L, p)[0].numpy()
    np.testing.assert_allclose(gp, tgp, rtol=1e-9, atol=1e-10 * np.abs(tgp).max())
